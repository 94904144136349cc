// Device-side bodies of the immersed-boundary transfer kernels, shared by
// the single-lattice kernels (transfer.cu) and the batched serving kernels
// (serve.cu). Transfer kernels (Sec. 2.3 of arXiv:1704.04551):
//   spread       g(x) += F_k delta(x - X_k)          (Eq. ibmForceSpread)
//   interpolate  U_k = sum_x u(x) delta(x - X_k),    (Eq. ibmVelocityInterpret)
//                then X_k += U_k (explicit advection, dt = 1, FP64)
// with delta(x) = phi(x) phi(y) phi(z), phi(r) = (1 + cos(pi r / 2)) / 4 for
// |r| <= 2 (Eq. deltaPhiSimple). The 4-point stencil of a marker at X is the
// nodes floor(X)-1 .. floor(X)+2 on each axis; nodes inside walls or the
// tube's solid are skipped (no renormalisation). Periodic axes wrap.
//
// Positions are FP64, but these kernels read the per-marker stencil cache
// (floor(X) as integers, X - floor(X) rounded once to FP32), which the
// interpolation kernel refreshes right after advecting each marker; the only
// FP64 arithmetic left is that advection.
//
// One thread block per marker group (a body, or a run of tracers), four
// threads per marker: lane a handles the stencil's x offset a, so the four
// read or write consecutive words, and the y/z weights are computed once and
// shared by shuffles. The block bounds the group's stencils with a box; when
// the box fits in shared memory (BOX_CELLS cells):
//   spreading accumulates there in 32-bit fixed point (native integer
//   shared-memory atomics; the sum does not depend on the order of the
//   additions) with a scale chosen from the group's largest force so that no
//   cell can overflow, then adds the box's nonzero cells to global memory
//   (one float4 atomic each);
//   interpolation loads the box of velocities once and gathers from shared
//   memory.
// Larger boxes (scattered tracers, very large bodies) fall back to
// per-marker global float4 atomics / gathers. The box of each group is
// computed by the spread kernel and reused by the interpolation of the same
// step (markers do not move in between).
#pragma once
#include <climits>

#include "common.cuh"

namespace ibm {

namespace xfer_detail {

constexpr int XFER_THREADS = 512;   // two blocks per SM (shared-memory box), 32 warps
constexpr int BOX_CELLS = 8192;     // 3 words per cell: 96 KiB of shared memory

__device__ __forceinline__ float phi(float r) { return 0.25f * (1.0f + cospif(0.5f * r)); }

// Stencil of marker k as seen by lane a of its 4-lane group: first node
// (unwrapped) on each axis, this lane's x weight and the four y and z
// weights (computed one per lane and shared by shuffles). All 32 lanes of
// the warp must call this (inactive groups pass any valid k).
struct LaneStencil {
  int bx, by, bz;
  float wx;           // weight of node bx + a
  float wy[4], wz[4];
};
// The stencil cache of one marker as read from global memory (the
// interpolation loads the next pass's entries while the current pass
// gathers, so that a pass does not wait for its own loads).
struct RawStencil {
  int c[3];
  float f[3];
};
__device__ __forceinline__ void load_raw(const MarkersDev& m, int k, RawStencil& r) {
  const size_t M = (size_t)m.M;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    r.c[q] = m.cell[q * M + k];
    r.f[q] = m.frac[q * M + k];
  }
}
__device__ __forceinline__ void lane_stencil(const RawStencil& r, int a, LaneStencil& s) {
  s.bx = r.c[0] - 1;
  s.by = r.c[1] - 1;
  s.bz = r.c[2] - 1;
  // node b + a sits at distance (a - 1) - frac from X
  s.wx = phi((float)(a - 1) - r.f[0]);
  const float wy_own = phi((float)(a - 1) - r.f[1]), wz_own = phi((float)(a - 1) - r.f[2]);
  const int base = threadIdx.x & 28;  // first lane of this 4-lane group within the warp
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    s.wy[b] = __shfl_sync(0xffffffffu, wy_own, base + b);
    s.wz[b] = __shfl_sync(0xffffffffu, wz_own, base + b);
  }
}

// wrap / range handling of a stencil row (y, z) for the geometry; false if
// the row is solid (outside the walls or the tube, or out of range)
template <int GEOM>
__device__ __forceinline__ bool fluid_row(const LatticeDev& L, int& y, int& z) {
  if (GEOM != GEOM_TUBE) z = wrapi(z, L.nz);
  if (GEOM == GEOM_PERIODIC) {
    y = wrapi(y, L.ny);
    return true;
  }
  return !solid_yz(L, y, z);
}

// Tiles (at most 2 per axis) covered by a stencil that starts at node b on
// an axis of n nodes with tile shift sh; periodic axes wrap, others clip.
template <bool PERIODIC>
__device__ __forceinline__ int axis_tiles(int b, int n, int sh, int t[2]) {
  int v = PERIODIC ? wrapi(b, n) : b;
  int cnt = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a, ++v) {
    if (PERIODIC && v >= n) v -= n;
    if (!PERIODIC && (unsigned)v >= (unsigned)n) continue;
    const int q = v >> sh;
    if (cnt == 0 || t[cnt - 1] != q) { if (cnt < 2) t[cnt++] = q; }
  }
  return cnt;
}

// Mark the (at most 8) tiles covered by a marker's stencil. Markers of a
// group are numbered along a space-filling curve, so a marker whose tile set
// equals that of the marker handled by the previous 4-lane group of the warp
// skips its stores.
template <int GEOM>
__device__ __forceinline__ void mark_tiles(const LatticeDev& L, int bx, int by, int bz, bool active) {
  int tx[2] = {-1, -1}, ty[2] = {-1, -1}, tz[2] = {-1, -1};
  const int nx_ = axis_tiles<true>(bx, L.nx, TILE_X_SHIFT, tx);
  const int ny_ = GEOM == GEOM_PERIODIC ? axis_tiles<true>(by, L.ny, TILE_Y_SHIFT, ty)
                                        : axis_tiles<false>(by, L.ny, TILE_Y_SHIFT, ty);
  const int nz_ = GEOM != GEOM_TUBE ? axis_tiles<true>(bz, L.nz, TILE_Z_SHIFT, tz)
                                    : axis_tiles<false>(bz, L.nz, TILE_Z_SHIFT, tz);
  // same tile set as the previous 4-lane group in the warp?
  const int src = ((int)(threadIdx.x & 31) - 4) & 31;
  bool same = __shfl_sync(0xffffffffu, (int)active, src) != 0 && (threadIdx.x & 31) >= 4;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    same &= __shfl_sync(0xffffffffu, tx[q], src) == tx[q];
    same &= __shfl_sync(0xffffffffu, ty[q], src) == ty[q];
    same &= __shfl_sync(0xffffffffu, tz[q], src) == tz[q];
  }
  if (!active || same) return;
  for (int c = 0; c < nz_; ++c)
    for (int b = 0; b < ny_; ++b)
      for (int a = 0; a < nx_; ++a) L.flags[tx[a] + L.ntx * (ty[b] + L.nty * tz[c])] = 1;
}

// Tiles covered by nodes lo .. lo + n - 1 (unwrapped) of an axis of `size`
// nodes with tile shift sh, as at most two ranges [t0, t1] of tile indices;
// periodic axes wrap, others clip. Returns the number of ranges.
template <bool PERIODIC>
__device__ __forceinline__ int axis_tile_ranges(int lo, int n, int size, int sh, int2 r[2]) {
  if (PERIODIC) {
    if (n >= size) {
      r[0] = make_int2(0, (size - 1) >> sh);
      return 1;
    }
    const int s = wrapi(lo, size), e = s + n - 1;
    if (e < size) {
      r[0] = make_int2(s >> sh, e >> sh);
      return 1;
    }
    r[0] = make_int2(s >> sh, (size - 1) >> sh);
    r[1] = make_int2(0, (e - size) >> sh);
    return 2;
  }
  const int s = max(lo, 0), e = min(lo + n - 1, size - 1);
  if (s > e) return 0;
  r[0] = make_int2(s >> sh, e >> sh);
  return 1;
}

// Mark every tile that intersects the box [lo, lo + dims) by the whole
// block: a superset of the tiles the group's stencils touch, at a cost of a
// few stores per group.
template <int GEOM>
__device__ __forceinline__ void mark_box_tiles(const LatticeDev& L, int4 lo, int4 dims) {
  int2 rx[2], ry[2], rz[2];
  const int nrx = axis_tile_ranges<true>(lo.x, dims.x, L.nx, TILE_X_SHIFT, rx);
  const int nry = GEOM == GEOM_PERIODIC ? axis_tile_ranges<true>(lo.y, dims.y, L.ny, TILE_Y_SHIFT, ry)
                                        : axis_tile_ranges<false>(lo.y, dims.y, L.ny, TILE_Y_SHIFT, ry);
  const int nrz = GEOM != GEOM_TUBE ? axis_tile_ranges<true>(lo.z, dims.z, L.nz, TILE_Z_SHIFT, rz)
                                    : axis_tile_ranges<false>(lo.z, dims.z, L.nz, TILE_Z_SHIFT, rz);
  for (int iz = 0; iz < nrz; ++iz)
    for (int iy = 0; iy < nry; ++iy)
      for (int ix = 0; ix < nrx; ++ix) {
        const int ax = rx[ix].y - rx[ix].x + 1, ay = ry[iy].y - ry[iy].x + 1, az = rz[iz].y - rz[iz].x + 1;
        for (int i = threadIdx.x; i < ax * ay * az; i += blockDim.x) {
          const int tx = rx[ix].x + i % ax, ty = ry[iy].x + (i / ax) % ay, tz = rz[iz].x + i / (ax * ay);
          L.flags[tx + L.ntx * (ty + L.nty * tz)] = 1;
        }
      }
}

// Bounding box of the group's stencil nodes (unwrapped coordinates) and the
// group's largest force component.
__device__ inline void group_box(const MarkersDev& m, const MarkerGroup& G, int4& lo, int4& dims, float& fmax) {
  __shared__ int s_lo[3], s_hi[3];
  __shared__ unsigned s_fmax;
  if (threadIdx.x < 3) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
  }
  if (threadIdx.x == 0) s_fmax = 0u;
  __syncthreads();
  const size_t M = (size_t)m.M;
  int lx = INT_MAX, ly = INT_MAX, lz = INT_MAX, hx = INT_MIN, hy = INT_MIN, hz = INT_MIN;
  float fm = 0.f;
  for (int k = G.first + threadIdx.x; k < G.first + G.count; k += blockDim.x) {
    const int cx_ = m.cell[k], cy_ = m.cell[M + k], cz_ = m.cell[2 * M + k];
    lx = min(lx, cx_); ly = min(ly, cy_); lz = min(lz, cz_);
    hx = max(hx, cx_); hy = max(hy, cy_); hz = max(hz, cz_);
    const float4 F = m.F[k];
    fm = fmaxf(fm, fmaxf(fabsf(F.x), fmaxf(fabsf(F.y), fabsf(F.z))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lx = min(lx, __shfl_xor_sync(0xffffffffu, lx, o));
    ly = min(ly, __shfl_xor_sync(0xffffffffu, ly, o));
    lz = min(lz, __shfl_xor_sync(0xffffffffu, lz, o));
    hx = max(hx, __shfl_xor_sync(0xffffffffu, hx, o));
    hy = max(hy, __shfl_xor_sync(0xffffffffu, hy, o));
    hz = max(hz, __shfl_xor_sync(0xffffffffu, hz, o));
    fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&s_lo[0], lx); atomicMin(&s_lo[1], ly); atomicMin(&s_lo[2], lz);
    atomicMax(&s_hi[0], hx); atomicMax(&s_hi[1], hy); atomicMax(&s_hi[2], hz);
    atomicMax(&s_fmax, __float_as_uint(fm));  // non-negative floats order as their bits
  }
  __syncthreads();
  const long long ex = (long long)s_hi[0] - s_lo[0] + 4, ey = (long long)s_hi[1] - s_lo[1] + 4,
                  ez = (long long)s_hi[2] - s_lo[2] + 4;
  lo = make_int4(s_lo[0] - 1, s_lo[1] - 1, s_lo[2] - 1, 0);
  const bool fits = ex > 0 && ey > 0 && ez > 0 && ex * ey * ez <= BOX_CELLS;
  dims = make_int4(fits ? (int)ex : 0, fits ? (int)ey : 0, fits ? (int)ez : 0, fits ? 1 : 0);
  fmax = __uint_as_float(s_fmax);
}

// Round-to-nearest-even of |v| <= 2^22 to an integer with one full-rate add:
// v + 1.5 * 2^23 has a fixed exponent, so its low mantissa bits hold
// round(v) + 2^22 (the float-to-int conversion unit runs at a quarter of the
// FP32 rate).
__device__ __forceinline__ int to_fixed(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }


// Lane mapping of a row-by-row sweep over a box whose rows hold dx cells:
// rows shorter than a warp are packed rpw to a warp (lane -> sub-row sub,
// offset ax); longer rows take one warp each, lanes striding by 32.
struct RowSweep {
  int rpw, sub, ax;
  bool on;
};
__device__ __forceinline__ RowSweep row_sweep(int dx) {
  const int lane = threadIdx.x & 31;
  RowSweep w;
  if (dx >= 32 || dx <= 0) {
    w.rpw = 1; w.sub = 0; w.ax = lane; w.on = true;
  } else {
    w.rpw = 32 / dx;
    w.sub = lane / dx;
    w.ax = lane - w.sub * dx;
    w.on = w.sub < w.rpw;
  }
  return w;
}

}  // namespace xfer_detail
using namespace xfer_detail;

// Spreading of one marker group by the whole thread block; box_out receives
// the group's stencil box (origin, size) for the interpolation of this step.
template <int GEOM>
__device__ __forceinline__ void spread_group(const LatticeDev& L, const MarkersDev& m, const MarkerGroup G,
                                             int4* box_out, int* ibox) {
  int4 lo, dims;
  float fmax;
  group_box(m, G, lo, dims, fmax);  // synchronises
  if (threadIdx.x == 0) {
    box_out[0] = lo;
    box_out[1] = dims;
  }
  const bool any_force = fmax > 0.f;
  const bool in_smem = dims.w != 0;
  // touched tiles: from the box when it fits, else marker by marker below
  if (in_smem) mark_box_tiles<GEOM>(L, lo, dims);
  const int vol = dims.x * dims.y * dims.z;
  // Fixed-point scale: a contribution is at most fmax / 8 (delta <= 1/8) and
  // a cell's sum at most count * fmax / 8; S keeps contributions below 2^22
  // (converted exactly by to_fixed) and sums below 2^30.
  const float S = any_force ? fminf(33554432.0f, 8589934592.0f / (float)G.count) / fmax : 0.f;
  if (in_smem && any_force) {
    for (int i = threadIdx.x; i < 3 * vol; i += blockDim.x) ibox[i] = 0;
    __syncthreads();
  }
  const int a = threadIdx.x & 3;
  // whole warps iterate together (shuffles inside)
  for (int j0 = 0; j0 < G.count; j0 += blockDim.x >> 2) {
    if (j0 + ((threadIdx.x >> 5) << 3) >= G.count) continue;  // the whole warp is past the group's end
    if (in_smem && !any_force) break;
    const int j = j0 + (threadIdx.x >> 2);
    const bool active = j < G.count;
    const int k = G.first + (active ? j : 0);
    RawStencil r;
    load_raw(m, k, r);
    LaneStencil s;
    lane_stencil(r, a, s);
    if (!in_smem) mark_tiles<GEOM>(L, s.bx, s.by, s.bz, active && a == 0);
    if (!active || !any_force) continue;
    const float4 F = m.F[k];
    if (in_smem) {
      const int li0 = (s.bx - lo.x + a) + dims.x * ((s.by - lo.y) + dims.y * (s.bz - lo.z));
      const float fx = F.x * S * s.wx, fy = F.y * S * s.wx, fz = F.z * S * s.wx;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float w = s.wy[b] * s.wz[c];
          const int li = li0 + dims.x * (b + dims.y * c);
          atomicAdd(ibox + li, to_fixed(fx * w));
          atomicAdd(ibox + vol + li, to_fixed(fy * w));
          atomicAdd(ibox + 2 * vol + li, to_fixed(fz * w));
        }
    } else {
      const int x = wrapi(s.bx + a, L.nx);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int y = s.by + b, z = s.bz + c;
          if (!fluid_row<GEOM>(L, y, z)) continue;
          const float w = s.wx * s.wy[b] * s.wz[c];
          atomicAdd(L.g + L.nx * (y + L.ny * z) + x, make_float4(F.x * w, F.y * w, F.z * w, 0.f));
        }
      }
    }
  }
  if (!in_smem || !any_force) return;
  __syncthreads();
  // add the nonzero cells of the box to the lattice, row by row
  const float inv = 1.0f / S;
  const int nrows = dims.y * dims.z;
  const int nwarps = blockDim.x >> 5;
  const RowSweep sw = row_sweep(dims.x);
  const int xw0 = wrapi(lo.x, L.nx);
  for (int ax = sw.ax; sw.on && ax < dims.x; ax += 32) {
    int x = xw0 + ax;
    if (x >= L.nx) x = (ax < L.nx) ? x - L.nx : wrapi(x, L.nx);
    for (int r = (threadIdx.x >> 5) * sw.rpw + sw.sub; r < nrows; r += nwarps * sw.rpw) {
      const int li = r * dims.x + ax;
      const int qx = ibox[li], qy = ibox[vol + li], qz = ibox[2 * vol + li];
      if ((qx | qy | qz) == 0) continue;
      int y = lo.y + r % dims.y, z = lo.z + r / dims.y;
      if (!fluid_row<GEOM>(L, y, z)) continue;
      atomicAdd(L.g + (size_t)L.nx * (y + L.ny * z) + x,
                make_float4((float)qx * inv, (float)qy * inv, (float)qz * inv, 0.f));
    }
  }
}

// Interpolation and advection of one marker group by the whole thread block.
template <int GEOM>
__device__ __forceinline__ void interpolate_group(const LatticeDev& L, const MarkersDev& m, const MarkerGroup G,
                                                  const int4* box_in, float* box) {
  const int4 lo = box_in[0], dims = box_in[1];
  const size_t M = (size_t)m.M;
  const bool in_smem = dims.w != 0;
  const int vol = dims.x * dims.y * dims.z;
  const int a = threadIdx.x & 3;
  const int pass = blockDim.x >> 2;            // markers per pass
  const int slot = threadIdx.x >> 2;           // this lane's marker within a pass
  const int wfirst = (threadIdx.x >> 5) << 3;  // first marker of this warp within a pass
  const bool moves = !(G.flags & GROUP_FIXED);
  // the first pass's stencil cache is loaded while the velocity box is
  RawStencil nxt;
  if (wfirst < G.count) load_raw(m, G.first + (slot < G.count ? slot : 0), nxt);
  if (in_smem) {
    // load the box of velocities row by row; solid rows contribute zero
    // one warp per box row, four rows in flight per lane (the loads are
    // latency-bound: the rows are short)
    constexpr int RIF = 4;
    const int nrows = dims.y * dims.z;
    const int nwarps = blockDim.x >> 5;
    const RowSweep sw = row_sweep(dims.x);
    const int rstep = nwarps * sw.rpw;
    const int xw0 = wrapi(lo.x, L.nx);
    for (int ax = sw.ax; sw.on && ax < dims.x; ax += 32) {
      int x = xw0 + ax;
      if (x >= L.nx) x = (ax < L.nx) ? x - L.nx : wrapi(x, L.nx);
      for (int r0 = (threadIdx.x >> 5) * sw.rpw + sw.sub; r0 < nrows; r0 += RIF * rstep) {
        float4 u[RIF];
#pragma unroll
        for (int q = 0; q < RIF; ++q) {
          const int r = r0 + q * rstep;
          u[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          int y = lo.y + r % dims.y, z = lo.z + r / dims.y;
          if (r < nrows && fluid_row<GEOM>(L, y, z)) {
            const size_t gi = (size_t)L.nx * (y + L.ny * z) + x;
            u[q] = L.uw[gi];
            L.g[gi] = make_float4(0.f, 0.f, 0.f, 0.f);  // consumed by this step's collision
          }
        }
#pragma unroll
        for (int q = 0; q < RIF; ++q) {
          const int r = r0 + q * rstep;
          if (r >= nrows) continue;
          const int li = r * dims.x + ax;
          box[li] = u[q].x;
          box[vol + li] = u[q].y;
          box[2 * vol + li] = u[q].z;
        }
      }
    }
    __syncthreads();
  }
  // whole warps iterate together (shuffles inside); a warp stops at the
  // first pass that lies entirely past the group's end
  for (int j0 = 0; j0 + wfirst < G.count; j0 += pass) {
    const int j = j0 + slot;
    const bool active = j < G.count;
    const int k = G.first + (active ? j : 0);
    // this lane's coordinate (advection) and the next pass's stencil cache
    // are loaded before the gather
    const size_t off = (size_t)a * M + k;
    double Xo = 0.0;
    if (active && moves && a < 3) Xo = m.X[off];
    const RawStencil cur = nxt;
    if (j0 + pass + wfirst < G.count) {
      const int jn = j + pass;
      load_raw(m, G.first + (jn < G.count ? jn : 0), nxt);
    }
    LaneStencil s;
    lane_stencil(cur, a, s);
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (in_smem) {
      const int li0 = (s.bx - lo.x + a) + dims.x * ((s.by - lo.y) + dims.y * (s.bz - lo.z));
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float w = s.wy[b] * s.wz[c];
          const int li = li0 + dims.x * (b + dims.y * c);
          ux = fmaf(w, box[li], ux);
          uy = fmaf(w, box[vol + li], uy);
          uz = fmaf(w, box[2 * vol + li], uz);
        }
    } else {
      const int x = wrapi(s.bx + a, L.nx);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int y = s.by + b, z = s.bz + c;
          if (!fluid_row<GEOM>(L, y, z)) continue;
          const float w = s.wy[b] * s.wz[c];
          const float4 u = L.uw[L.nx * (y + L.ny * z) + x];
          L.g[L.nx * (y + L.ny * z) + x] = make_float4(0.f, 0.f, 0.f, 0.f);  // consumed by the collision
          ux = fmaf(w, u.x, ux);
          uy = fmaf(w, u.y, uy);
          uz = fmaf(w, u.z, uz);
        }
      }
    }
    ux *= s.wx; uy *= s.wx; uz *= s.wx;
    // sum the four x columns of the stencil
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      ux += __shfl_xor_sync(0xffffffffu, ux, o);
      uy += __shfl_xor_sync(0xffffffffu, uy, o);
      uz += __shfl_xor_sync(0xffffffffu, uz, o);
    }
    if (!active) continue;
    if (a == 0) m.U[k] = make_float4(ux, uy, uz, 0.f);
    if (a < 3 && moves) {
      // advection of one coordinate per lane (FP64), then its stencil cache
      const float ua = a == 0 ? ux : (a == 1 ? uy : uz);
      const double Xn = Xo + (double)ua;
      m.X[off] = Xn;
      cache_coord(m, off, Xn);
    }
  }
}

}  // namespace ibm

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
// Delta weights: with f = X - floor(X) in [0, 1) and t = pi f / 2, the four
// nodes sit at r = -1-f, -f, 1-f, 2-f, where cos(pi r / 2) is -sin t,
// cos t, sin t, -cos t. One sine/cosine pair per axis gives all four
// weights: (1 - sin t)/4, (1 + cos t)/4, (1 + sin t)/4, (1 - cos t)/4.
//
// Positions are FP64, but these kernels read the per-marker stencil cache
// (floor(X) as integers, X - floor(X) rounded once to FP32), which the
// interpolation kernel refreshes right after advecting each marker; the only
// FP64 arithmetic left is that advection.
//
// One thread block per marker group (a body, or a run of tracers). Launches
// of many groups (several blocks per SM) take one thread per marker: a
// thread computes its marker's 12 weights once and visits the 64 stencil
// nodes itself; which marker a lane takes is chosen so that a warp's
// shared-memory accesses fall in distinct banks (see Residues below).
// Launches of few groups are bound by the latency of one block's passes:
// they take larger blocks and four lanes per marker, lane a visiting the
// stencil's x column a (the *_lanes functions). The block bounds the
// group's stencils with a box; when the box fits in shared memory
// (BOX_CELLS cells):
//   spreading accumulates there in 32-bit fixed point (native integer
//   shared-memory atomics; the sum does not depend on the order of the
//   additions) with a scale chosen from the group's largest force so that no
//   cell can overflow, then adds the box's nonzero cells to global memory
//   (one float4 atomic each);
//   interpolation loads the box of velocities (float4 per cell, so that one
//   16-byte shared load serves a node) once, with asynchronous copies, and
//   gathers from shared memory; the same sweep clears the force density the
//   collision has consumed.
// Larger boxes (scattered tracers, very large bodies) fall back to
// per-marker global float4 atomics / gathers. The box of each group is
// computed by the spread kernel and reused by the interpolation of the same
// step (markers do not move in between; a marker found outside the box
// takes the per-marker path).
#pragma once
#include <climits>

#include "common.cuh"

namespace ibm {

namespace xfer_detail {

constexpr int XFER_THREADS = 352;   // 11 warps
constexpr int BOX_CELLS = 6144;     // shared-memory box limit (cells)
constexpr int XFER_GROUP_MAX = 1024;  // markers per group (records in shared memory)
constexpr int XFER_PER_THREAD = (XFER_GROUP_MAX + XFER_THREADS - 1) / XFER_THREADS;
constexpr int RESIDUE_BYTES = 512;   // the counting sort's counters (struct Residues)
// Launches of fewer groups than this take the four-lanes-per-marker
// functions in blocks of LANE_THREADS: with at most a few blocks per SM the
// time of one block's passes decides, not the issue rate of many.
constexpr int LANE_MAX_GROUPS = 512;
constexpr int LANE_THREADS = 1024;
// fixed-point sums [3][vol], two float4 records per marker, counters
constexpr int SPREAD_SMEM =
    3 * BOX_CELLS * (int)sizeof(int) + 2 * XFER_GROUP_MAX * (int)sizeof(float4) + RESIDUE_BYTES;
// velocities [vol] float4
constexpr int INTERP_SMEM = BOX_CELLS * (int)sizeof(float4);
// fixed-point sums [3][vol] (four lanes per marker: no marker records)
constexpr int SPREAD_LANES_SMEM = 3 * BOX_CELLS * (int)sizeof(int);

// The four delta weights of one axis for a marker at fractional offset f.
__device__ __forceinline__ void axis_weights(float f, float w[4]) {
  float s, c;
  sincospif(0.5f * f, &s, &c);
  w[0] = fmaf(-0.25f, s, 0.25f);
  w[1] = fmaf(0.25f, c, 0.25f);
  w[2] = fmaf(0.25f, s, 0.25f);
  w[3] = fmaf(-0.25f, c, 0.25f);
}

// Weight of node a (0..3) of one axis: entry a of axis_weights, computed
// alone (a lane that handles one node of each x column).
__device__ __forceinline__ float axis_weight(float f, int a) {
  float s, c;
  sincospif(0.5f * f, &s, &c);
  return fmaf((a == 0 || a == 3) ? -0.25f : 0.25f, (a & 1) ? c : s, 0.25f);
}

// Stencil of one marker: first node (unwrapped) on each axis and the
// weights of its four nodes per axis.
struct Stencil {
  int bx, by, bz;
  float wx[4], wy[4], wz[4];
};
__device__ __forceinline__ void load_stencil(const MarkersDev& m, int k, Stencil& s) {
  const size_t M = (size_t)m.M;
  s.bx = m.cell[k] - 1;
  s.by = m.cell[M + k] - 1;
  s.bz = m.cell[2 * M + k] - 1;
  axis_weights(m.frac[k], s.wx);
  axis_weights(m.frac[M + k], s.wy);
  axis_weights(m.frac[2 * M + k], s.wz);
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
// equals that of the previous lane's marker skips its stores. All 32 lanes
// of the warp call this.
template <int GEOM>
__device__ __forceinline__ void mark_tiles(const LatticeDev& L, int bx, int by, int bz, bool active) {
  int tx[2] = {-1, -1}, ty[2] = {-1, -1}, tz[2] = {-1, -1};
  const int nx_ = axis_tiles<true>(bx, L.nx, TILE_X_SHIFT, tx);
  const int ny_ = GEOM == GEOM_PERIODIC ? axis_tiles<true>(by, L.ny, TILE_Y_SHIFT, ty)
                                        : axis_tiles<false>(by, L.ny, TILE_Y_SHIFT, ty);
  const int nz_ = GEOM != GEOM_TUBE ? axis_tiles<true>(bz, L.nz, TILE_Z_SHIFT, tz)
                                    : axis_tiles<false>(bz, L.nz, TILE_Z_SHIFT, tz);
  const int lane = threadIdx.x & 31;
  bool same = __shfl_up_sync(0xffffffffu, (int)active, 1) != 0 && lane >= 1;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    same &= __shfl_up_sync(0xffffffffu, tx[q], 1) == tx[q];
    same &= __shfl_up_sync(0xffffffffu, ty[q], 1) == ty[q];
    same &= __shfl_up_sync(0xffffffffu, tz[q], 1) == tz[q];
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

// round(a * b) for |a b| <= 2^22, with one fused multiply-add: a b + 1.5 2^23
// has a fixed exponent, so its low mantissa bits hold round(a b) + 2^22
// (the float-to-int conversion unit runs at a quarter of the FP32 rate).
__device__ __forceinline__ int fixed_mul(float a, float b) {
  return __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
}

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

// Row r of a box with dy rows per z layer as (iy, iz), without an integer
// division: for 0 <= r < BOX_CELLS the float quotient (r + 1/2)/dy lies at
// least 1/(2 dy) from an integer, far beyond its rounding error.
__device__ __forceinline__ void row_yz(int r, int dy, float inv_dy, int& iy, int& iz) {
  iz = (int)(((float)r + 0.5f) * inv_dy);
  iy = r - iz * dy;
}

// Wrapped x of box column ax (box origin x0 already wrapped into [0, nx)).
__device__ __forceinline__ int box_x(int xw0, int ax, int nx) {
  const int x = xw0 + ax;
  if (x < nx) return x;
  return (ax < nx) ? x - nx : wrapi(x, nx);
}

// Index in the box of a marker's first stencil node, or -1 if its 4^3
// stencil is not inside the box.
__device__ __forceinline__ int box_index(const MarkersDev& m, int k, int4 lo, int4 dims) {
  const size_t M = (size_t)m.M;
  const int ox = m.cell[k] - 1 - lo.x, oy = m.cell[M + k] - 1 - lo.y, oz = m.cell[2 * M + k] - 1 - lo.z;
  if (ox < 0 || oy < 0 || oz < 0 || ox + 4 > dims.x || oy + 4 > dims.y || oz + 4 > dims.z) return -1;
  return ox + dims.x * (oy + dims.y * oz);
}

// Lane assignment without shared-memory bank conflicts. Every shared access
// of a marker's stencil is at box index li0 + (a fixed offset per node), so
// 32 markers whose li0 differ modulo 32 hit 32 distinct banks with 4-byte
// accesses (the spreading atomics) and, 8 by 8, distinct bank quads with
// 16-byte ones (the velocity gather). The group's markers are counted by
// li0 mod 32 (a counting sort in shared memory); lane r of a warp then takes
// the w-th marker of residue r. A marker's lane does not change any sum: the
// fixed-point atomics are order-independent and each gather is one thread's.
struct Residues {
  int cnt[32], start[32], cur[32];
  int most;
};
static_assert(sizeof(Residues) <= RESIDUE_BYTES, "counters");
// after the counts: exclusive prefix (start, cursor) and the largest class
__device__ __forceinline__ void residue_scan(Residues& R) {
  if (threadIdx.x < 32) {
    const int c = R.cnt[threadIdx.x];
    int incl = c, mx = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)threadIdx.x >= o) incl += v;
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    R.start[threadIdx.x] = incl - c;
    R.cur[threadIdx.x] = incl - c;
    if (threadIdx.x == 0) R.most = mx;
  }
}

}  // namespace xfer_detail
using namespace xfer_detail;

// Force of one marker added to the lattice with global float4 atomics
// (groups whose box does not fit in shared memory). Kept out of line: it is
// the rare path.
template <int GEOM>
__device__ __noinline__ void scatter_global(const LatticeDev& L, const Stencil& s, float4 F) {
  int xs[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) xs[a] = wrapi(s.bx + a, L.nx);
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
      int y = s.by + b, z = s.bz + c;
      if (!fluid_row<GEOM>(L, y, z)) continue;
      const float wyz = s.wy[b] * s.wz[c];
      float4* row = L.g + (size_t)L.nx * (y + L.ny * z);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = s.wx[a] * wyz;
        atomicAdd(row + xs[a], make_float4(F.x * w, F.y * w, F.z * w, 0.f));
      }
    }
  }
}

// Adds one marker's force, already multiplied by the fixed-point scale, to
// the box: li0 is the box index of its first stencil node, f its fractional
// offsets (the weights), vol the box's cells per component.
__device__ __forceinline__ void scatter_marker(int* ibox, int vol, int4 dims, int li0, float fx, float fy, float fz,
                                               float Fx, float Fy, float Fz) {
  float wx[4], wy[4], wz[4];
  axis_weights(fx, wx);
  axis_weights(fy, wy);
  axis_weights(fz, wz);
  float ax_[4], ay_[4], az_[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ax_[a] = Fx * wx[a];
    ay_[a] = Fy * wx[a];
    az_[a] = Fz * wx[a];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float wyz = wy[b] * wz[c];
      int* p = ibox + li0 + dims.x * (b + dims.y * c);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        atomicAdd(p + a, fixed_mul(ax_[a], wyz));
        atomicAdd(p + vol + a, fixed_mul(ay_[a], wyz));
        atomicAdd(p + 2 * vol + a, fixed_mul(az_[a], wyz));
      }
    }
}

// Adds the nonzero cells of a fixed-point box (1/inv units) to L.g, row by
// row (one float4 atomic per cell).
template <int GEOM>
__device__ __forceinline__ void flush_box(const LatticeDev& L, int4 lo, int4 dims, const int* ibox, float inv) {
  const int vol = dims.x * dims.y * dims.z;
  const int nrows = dims.y * dims.z;
  const int nwarps = blockDim.x >> 5;
  const RowSweep sw = row_sweep(dims.x);
  const float inv_dy = 1.0f / (float)dims.y;
  const int xw0 = wrapi(lo.x, L.nx);
  for (int ax = sw.ax; sw.on && ax < dims.x; ax += 32) {
    const int x = box_x(xw0, ax, L.nx);
    for (int r = (threadIdx.x >> 5) * sw.rpw + sw.sub; r < nrows; r += nwarps * sw.rpw) {
      const int i = r * dims.x + ax;
      const int qx = ibox[i], qy = ibox[vol + i], qz = ibox[2 * vol + i];
      if ((qx | qy | qz) == 0) continue;
      int iy, iz;
      row_yz(r, dims.y, inv_dy, iy, iz);
      int y = lo.y + iy, z = lo.z + iz;
      if (!fluid_row<GEOM>(L, y, z)) continue;
      atomicAdd(L.g + (size_t)L.nx * (y + L.ny * z) + x,
                make_float4((float)qx * inv, (float)qy * inv, (float)qz * inv, 0.f));
    }
  }
}

// Issues the load of the box of velocities (row by row, asynchronous 16-byte
// copies; solid rows are written as zero) and clears the force density
// there (consumed by this step's collision). The copies complete at
// velocity_box_wait() followed by a barrier.
template <int GEOM>
__device__ __forceinline__ void velocity_box_async(const LatticeDev& L, int4 lo, int4 dims, float4* vbox) {
  const int nrows = dims.y * dims.z;
  const int nwarps = blockDim.x >> 5;
  const RowSweep sw = row_sweep(dims.x);
  const int rstep = nwarps * sw.rpw;
  const float inv_dy = 1.0f / (float)dims.y;
  const int xw0 = wrapi(lo.x, L.nx);
  for (int ax = sw.ax; sw.on && ax < dims.x; ax += 32) {
    const int x = box_x(xw0, ax, L.nx);
    for (int r = (threadIdx.x >> 5) * sw.rpw + sw.sub; r < nrows; r += rstep) {
      int iy, iz;
      row_yz(r, dims.y, inv_dy, iy, iz);
      int y = lo.y + iy, z = lo.z + iz;
      float4* dst = vbox + r * dims.x + ax;
      if (fluid_row<GEOM>(L, y, z)) {
        const size_t gi = (size_t)L.nx * (y + L.ny * z) + x;
        const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(L.uw + gi) : "memory");
        L.g[gi] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        *dst = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void velocity_box_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Velocity at a marker whose 4^3 stencil lies in the box (first node at
// box offsets ox, oy, oz), gathered from the shared-memory box.
__device__ __forceinline__ float3 box_gather(const float4* vbox, int4 dims, const Stencil& st, int ox, int oy, int oz) {
  const int li0 = ox + dims.x * (oy + dims.y * oz);
  float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4* p = vbox + li0 + dims.x * (b + dims.y * c);
      const float4 v0 = p[0], v1 = p[1], v2 = p[2], v3 = p[3];
      const float rx = fmaf(st.wx[3], v3.x, fmaf(st.wx[2], v2.x, fmaf(st.wx[1], v1.x, st.wx[0] * v0.x)));
      const float ry = fmaf(st.wx[3], v3.y, fmaf(st.wx[2], v2.y, fmaf(st.wx[1], v1.y, st.wx[0] * v0.y)));
      const float rz = fmaf(st.wx[3], v3.z, fmaf(st.wx[2], v2.z, fmaf(st.wx[1], v1.z, st.wx[0] * v0.z)));
      const float wyz = st.wy[b] * st.wz[c];
      ux = fmaf(wyz, rx, ux);
      uy = fmaf(wyz, ry, uy);
      uz = fmaf(wyz, rz, uz);
    }
  return make_float3(ux, uy, uz);
}

// Spreading of one marker group by the whole thread block; box_out receives
// the group's stencil box (origin, size) for the interpolation of this step.
// smem: SPREAD_SMEM bytes (fixed-point box, then the marker records).
template <int GEOM>
__device__ __forceinline__ void spread_group(const LatticeDev& L, const MarkersDev& m, const MarkerGroup G,
                                             int4* box_out, unsigned char* smem) {
  int4 lo, dims;
  float fmax;
  group_box(m, G, lo, dims, fmax);  // synchronises
  if (threadIdx.x == 0) {
    box_out[0] = lo;
    box_out[1] = dims;
  }
  const bool any_force = fmax > 0.f;
  const bool in_smem = dims.w != 0;
  if (!in_smem) {
    // per-marker global atomics; touched tiles marker by marker (whole warps
    // iterate together: shuffles in mark_tiles)
    for (int j0 = 0; j0 < G.count; j0 += blockDim.x) {
      if (j0 + (int)(threadIdx.x & ~31u) >= G.count) break;
      const int j = j0 + threadIdx.x;
      const bool active = j < G.count;
      const int k = G.first + (active ? j : 0);
      Stencil s;
      load_stencil(m, k, s);
      mark_tiles<GEOM>(L, s.bx, s.by, s.bz, active);
      if (active && any_force) scatter_global<GEOM>(L, s, m.F[k]);
    }
    return;
  }
  mark_box_tiles<GEOM>(L, lo, dims);  // touched tiles: every tile the box meets
  if (!any_force) return;
  int* ibox = reinterpret_cast<int*>(smem);                                   // [3][vol]
  float4* rec = reinterpret_cast<float4*>(smem + 3 * BOX_CELLS * sizeof(int));  // [2][XFER_GROUP_MAX]
  Residues& R = *reinterpret_cast<Residues*>(rec + 2 * XFER_GROUP_MAX);
  const int vol = dims.x * dims.y * dims.z;
  const size_t M = (size_t)m.M;
  // Fixed-point scale: a contribution is at most fmax / 8 (delta <= 1/8) and
  // a cell's sum at most count * fmax / 8; S keeps contributions below 2^22
  // (converted exactly by fixed_mul) and sums below 2^30.
  const float S = fminf(33554432.0f, 8589934592.0f / (float)G.count) / fmax;
  for (int i = threadIdx.x; i < 3 * vol; i += blockDim.x) ibox[i] = 0;
  if (threadIdx.x < 32) R.cnt[threadIdx.x] = 0;
  __syncthreads();
  // markers by residue of their first node's box index
  int li[XFER_PER_THREAD];
#pragma unroll
  for (int q = 0; q < XFER_PER_THREAD; ++q) {
    const int j = threadIdx.x + q * blockDim.x;  // blockDim.x >= XFER_THREADS
    li[q] = j < G.count ? box_index(m, G.first + j, lo, dims) : -1;  // inside by construction of the box
    if (li[q] >= 0) atomicAdd(&R.cnt[li[q] & 31], 1);
  }
  __syncthreads();
  residue_scan(R);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < XFER_PER_THREAD; ++q) {
    if (li[q] < 0) continue;
    const int k = G.first + threadIdx.x + q * blockDim.x;
    const int pos = atomicAdd(&R.cur[li[q] & 31], 1);
    const float4 F = m.F[k];
    rec[pos] = make_float4(__int_as_float(li[q]), m.frac[k], m.frac[M + k], m.frac[2 * M + k]);
    rec[XFER_GROUP_MAX + pos] = make_float4(F.x * S, F.y * S, F.z * S, 0.f);
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int n = R.cnt[lane], st = R.start[lane];
    for (int w = threadIdx.x >> 5; w < R.most; w += nwarps) {
      if (w >= n) continue;
      const float4 A = rec[st + w], B = rec[XFER_GROUP_MAX + st + w];
      scatter_marker(ibox, vol, dims, __float_as_int(A.x), A.y, A.z, A.w, B.x, B.y, B.z);
    }
  }
  __syncthreads();
  flush_box<GEOM>(L, lo, dims, ibox, 1.0f / S);
}

// Velocity at one marker gathered from the lattice (groups whose box does
// not fit in shared memory, or a marker outside its group's box); with
// clear, the visited cells' force density is reset (consumed by the
// collision). Kept out of line: it is the rare path.
template <int GEOM>
__device__ __noinline__ float3 gather_global(const LatticeDev& L, const Stencil& s, bool clear) {
  int xs[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) xs[a] = wrapi(s.bx + a, L.nx);
  float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
      int y = s.by + b, z = s.bz + c;
      if (!fluid_row<GEOM>(L, y, z)) continue;
      const size_t rb = (size_t)L.nx * (y + L.ny * z);
      float rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 v = L.uw[rb + xs[a]];
        if (clear) L.g[rb + xs[a]] = make_float4(0.f, 0.f, 0.f, 0.f);
        rx = fmaf(s.wx[a], v.x, rx);
        ry = fmaf(s.wx[a], v.y, ry);
        rz = fmaf(s.wx[a], v.z, rz);
      }
      const float w = s.wy[b] * s.wz[c];
      ux = fmaf(w, rx, ux);
      uy = fmaf(w, ry, uy);
      uz = fmaf(w, rz, uz);
    }
  }
  return make_float3(ux, uy, uz);
}

// Interpolation and advection of one marker group by the whole thread block:
// the velocity box is loaded once, then each thread gathers for its own
// markers (the bank conflicts of the gather cost less than sorting the
// markers by residue, which pays off for the atomics of the spreading only)
// and advects them. smem: INTERP_SMEM bytes (the velocity box).
template <int GEOM>
__device__ __forceinline__ void interpolate_group(const LatticeDev& L, const MarkersDev& m, const MarkerGroup G,
                                                  const int4* box_in, unsigned char* smem) {
  const int4 lo = box_in[0], dims = box_in[1];
  const size_t M = (size_t)m.M;
  const bool moves = !(G.flags & GROUP_FIXED);
  const bool in_box = dims.w != 0;
  float4* vbox = reinterpret_cast<float4*>(smem);  // [vol]
  if (in_box) {
    velocity_box_async<GEOM>(L, lo, dims, vbox);
    velocity_box_wait();
    __syncthreads();
  }
  for (int j = threadIdx.x; j < G.count; j += blockDim.x) {
    const int k = G.first + j;
    Stencil st;
    load_stencil(m, k, st);
    double Xo[3] = {0.0, 0.0, 0.0};
    if (moves)
#pragma unroll
      for (int a = 0; a < 3; ++a) Xo[a] = m.X[a * M + k];
    const int ox = st.bx - lo.x, oy = st.by - lo.y, oz = st.bz - lo.z;
    float3 u;
    if (in_box && ox >= 0 && oy >= 0 && oz >= 0 && ox + 4 <= dims.x && oy + 4 <= dims.y && oz + 4 <= dims.z)
      u = box_gather(vbox, dims, st, ox, oy, oz);
    else  // no box (every visited cell is cleared), or the stencil outside it
      u = gather_global<GEOM>(L, st, !in_box);
    m.U[k] = make_float4(u.x, u.y, u.z, 0.f);
    if (moves) {
      const float ua[3] = {u.x, u.y, u.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double Xn = Xo[a] + (double)ua[a];
        m.X[a * M + k] = Xn;
        cache_coord(m, a * M + k, Xn);
      }
    }
  }
}


// The stencil cache of one marker (first node and fractional offsets), as
// read by the four lanes that share the marker.
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

// Spreading of one marker group with four lanes per marker (launches of few
// groups); the same fixed-point contributions as spread_group, so the same
// sums. ibox: SPREAD_LANES_SMEM bytes.
template <int GEOM>
__device__ __forceinline__ void spread_group_lanes(const LatticeDev& L, const MarkersDev& m, const MarkerGroup G,
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
  const int vol = dims.x * dims.y * dims.z;
  const float S = any_force ? fminf(33554432.0f, 8589934592.0f / (float)G.count) / fmax : 0.f;  // as spread_group
  if (in_smem) {
    mark_box_tiles<GEOM>(L, lo, dims);
    if (!any_force) return;
    for (int i = threadIdx.x; i < 3 * vol; i += blockDim.x) ibox[i] = 0;
    __syncthreads();
  }
  const int a = threadIdx.x & 3;
  const int per_pass = blockDim.x >> 2;
  const int wfirst = (int)(threadIdx.x & ~31u) >> 2;  // first marker of this warp within a pass
  // whole warps iterate together (shuffles in mark_tiles)
  for (int j0 = 0; j0 + wfirst < G.count; j0 += per_pass) {
    const int j = j0 + (int)(threadIdx.x >> 2);
    const bool active = j < G.count;
    const int k = G.first + (active ? j : 0);
    RawStencil r;
    load_raw(m, k, r);
    const int bx = r.c[0] - 1, by = r.c[1] - 1, bz = r.c[2] - 1;
    // the four lanes of a marker share its tiles: only the first stores them
    if (!in_smem) mark_tiles<GEOM>(L, bx, by, bz, active);
    if (!active || !any_force) continue;
    const float wxa = axis_weight(r.f[0], a);
    float wy[4], wz[4];
    axis_weights(r.f[1], wy);
    axis_weights(r.f[2], wz);
    const float4 F = m.F[k];
    if (in_smem) {
      const float ax_ = F.x * S * wxa, ay_ = F.y * S * wxa, az_ = F.z * S * wxa;
      int* p0 = ibox + (bx - lo.x + a) + dims.x * ((by - lo.y) + dims.y * (bz - lo.z));
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float wyz = wy[b] * wz[c];
          int* p = p0 + dims.x * (b + dims.y * c);
          atomicAdd(p, fixed_mul(ax_, wyz));
          atomicAdd(p + vol, fixed_mul(ay_, wyz));
          atomicAdd(p + 2 * vol, fixed_mul(az_, wyz));
        }
    } else {
      const int x = wrapi(bx + a, L.nx);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int y = by + b, z = bz + c;
          if (!fluid_row<GEOM>(L, y, z)) continue;
          const float w = wxa * (wy[b] * wz[c]);
          atomicAdd(L.g + (size_t)L.nx * (y + L.ny * z) + x, make_float4(F.x * w, F.y * w, F.z * w, 0.f));
        }
    }
  }
  if (!in_smem) return;
  __syncthreads();
  flush_box<GEOM>(L, lo, dims, ibox, 1.0f / S);
}

// Interpolation and advection of one marker group with four lanes per
// marker (launches of few groups): lane a sums the stencil's x column a,
// the four partial sums meet by shuffles, and lanes 0..2 advect one
// coordinate each. The next pass's stencil cache is loaded before this
// pass gathers. smem: INTERP_SMEM bytes (the velocity box).
template <int GEOM>
__device__ __forceinline__ void interpolate_group_lanes(const LatticeDev& L, const MarkersDev& m,
                                                        const MarkerGroup G, const int4* box_in,
                                                        unsigned char* smem) {
  const int4 lo = box_in[0], dims = box_in[1];
  const size_t M = (size_t)m.M;
  const bool moves = !(G.flags & GROUP_FIXED);
  const bool in_box = dims.w != 0;
  float4* vbox = reinterpret_cast<float4*>(smem);  // [vol]
  const int a = threadIdx.x & 3;
  const int per_pass = blockDim.x >> 2;
  const int slot = threadIdx.x >> 2;
  const int wfirst = (int)(threadIdx.x & ~31u) >> 2;
  if (in_box) velocity_box_async<GEOM>(L, lo, dims, vbox);
  RawStencil nxt;
  if (wfirst < G.count) load_raw(m, G.first + (slot < G.count ? slot : 0), nxt);
  if (in_box) {
    velocity_box_wait();
    __syncthreads();
  }
  // whole warps iterate together (shuffles); a warp stops at the first pass
  // that lies entirely past the group's end
  for (int j0 = 0; j0 + wfirst < G.count; j0 += per_pass) {
    const int j = j0 + slot;
    const bool active = j < G.count;
    const int k = G.first + (active ? j : 0);
    const size_t off = (size_t)a * M + k;
    double Xo = 0.0;
    if (active && moves && a < 3) Xo = m.X[off];
    const RawStencil cur = nxt;
    if (j0 + per_pass + wfirst < G.count) {
      const int jn = j + per_pass;
      load_raw(m, G.first + (jn < G.count ? jn : 0), nxt);
    }
    const int bx = cur.c[0] - 1, by = cur.c[1] - 1, bz = cur.c[2] - 1;
    const float wxa = axis_weight(cur.f[0], a);
    float wy[4], wz[4];
    axis_weights(cur.f[1], wy);
    axis_weights(cur.f[2], wz);
    const int ox = bx - lo.x, oy = by - lo.y, oz = bz - lo.z;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (in_box && ox >= 0 && oy >= 0 && oz >= 0 && ox + 4 <= dims.x && oy + 4 <= dims.y && oz + 4 <= dims.z) {
      const float4* p0 = vbox + (ox + a) + dims.x * (oy + dims.y * oz);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float4 v = p0[dims.x * (b + dims.y * c)];
          const float wyz = wy[b] * wz[c];
          ux = fmaf(wyz, v.x, ux);
          uy = fmaf(wyz, v.y, uy);
          uz = fmaf(wyz, v.z, uz);
        }
    } else {  // no box (every visited cell is cleared), or the stencil outside it
      const int x = wrapi(bx + a, L.nx);
#pragma unroll 1
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int y = by + b, z = bz + c;
          if (!fluid_row<GEOM>(L, y, z)) continue;
          const size_t gi = (size_t)L.nx * (y + L.ny * z) + x;
          const float4 v = L.uw[gi];
          if (!in_box) L.g[gi] = make_float4(0.f, 0.f, 0.f, 0.f);
          const float wyz = wy[b] * wz[c];
          ux = fmaf(wyz, v.x, ux);
          uy = fmaf(wyz, v.y, uy);
          uz = fmaf(wyz, v.z, uz);
        }
    }
    ux *= wxa;
    uy *= wxa;
    uz *= wxa;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      ux += __shfl_xor_sync(0xffffffffu, ux, o);
      uy += __shfl_xor_sync(0xffffffffu, uy, o);
      uz += __shfl_xor_sync(0xffffffffu, uz, o);
    }
    if (!active) continue;
    if (a == 0) m.U[k] = make_float4(ux, uy, uz, 0.f);
    if (a < 3 && moves) {
      const double Xn = Xo + (double)(a == 0 ? ux : (a == 1 ? uy : uz));
      m.X[off] = Xn;
      cache_coord(m, off, Xn);
    }
  }
}

}  // namespace ibm

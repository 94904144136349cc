// Morse excluded volume between immersed bodies (Eq. morsePotential of
// arXiv:1704.04551, Sec. 2.2):
//   U = D0 (e^{-2 alpha (r - r0)} - 2 e^{-alpha (r - r0)}),  r < rc,
// between markers of different membrane or filament bodies; the force on a
// marker is F = -dU/dr d/r = 2 alpha D0 (e^2 - e) d/r, e = e^{-alpha (r - r0)},
// d its separation from the other marker (nearest image on periodic axes).
//
// A cell list rebuilt every step: bins at least rc wide (at most 2^26 of
// them), markers counted into bins with atomics, an exclusive prefix sum of
// the counts, markers scattered into bin order (wrapped position and owner
// body packed in a float4), then one thread per sorted marker gathers the
// forces of the markers in the 27 bins around its own and adds them to its
// marker force. Each bin also records whether all its markers belong to one
// body: a marker first loads the owners of its 27 neighbour bins (independent
// loads, kept as a bit mask) and then reads only the bins that hold markers
// of another body (a membrane's own vertices fill most bins around it). Positions come from the stencil cache (floor + FP32
// fraction), wrapped into the box on periodic axes, so separations are
// exact to FP32 rounding of a coordinate below the box size.
#include "common.cuh"
#include "internal.h"

namespace ibm {

namespace {

constexpr int MORSE_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;  // per thread: tiles of 8192 bins, at most 8192 tiles (2^26 bins)
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct Box {
  int n[3];
  int periodic[3];
};

__device__ __forceinline__ float wrapped_coord(const MarkersDev& m, const Box& B, int a, int k) {
  const size_t M = (size_t)m.M;
  int c = m.cell[a * M + k];
  if (B.periodic[a]) c = wrapi(c, B.n[a]);
  return (float)c + m.frac[a * M + k];
}

__device__ __forceinline__ int bin_coord(const MorseDev& P, int a, float x) {
  const int b = (int)floorf(x * P.inv_bs[a]);
  return min(max(b, 0), P.nb[a] - 1);
}

__global__ void k_morse_count(MorseDev P, MarkersDev m, Box B) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M || P.owner[k] < 0) return;
  int b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) b[a] = bin_coord(P, a, wrapped_coord(m, B, a, k));
  const int bin = b[0] + P.nb[0] * (b[1] + P.nb[1] * b[2]);
  P.bin_of[k] = bin;
  P.rank[k] = atomicAdd(P.count + bin, 1);
  P.bin_owner[bin] = -1;  // claimed again by the scatter (bins left empty keep a stale owner, never read as a range)
}

// exclusive scan of SCAN_ITEMS values per thread across the block; returns
// this thread's exclusive prefix and the block total
__device__ __forceinline__ int block_exclusive(int v, int& total) {
  __shared__ int warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  total = warp_tot[(blockDim.x >> 5) - 1];
  const int before = warp == 0 ? 0 : warp_tot[warp - 1];
  __syncthreads();  // warp_tot is reused by the next call
  return before + x - v;
}

// padded shared-memory index: conflict-free for both the coalesced
// (i = k * threads + t) and the per-thread contiguous (i = t * items + k) sweeps
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// tile-local exclusive prefix into start[], tile totals into block_sum[];
// the tile goes through shared memory so that global accesses coalesce
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(MorseDev P) {
  __shared__ int sh[SCAN_TILE + SCAN_TILE / 32];
  const int base = blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = k * SCAN_THREADS + threadIdx.x;
    sh[pad(i)] = base + i < P.n_bins ? P.count[base + i] : 0;
  }
  __syncthreads();
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = sh[pad(threadIdx.x * SCAN_ITEMS + k)];
    s += v[k];
  }
  int total;
  int run = block_exclusive(s, total);  // synchronises
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    sh[pad(threadIdx.x * SCAN_ITEMS + k)] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = k * SCAN_THREADS + threadIdx.x;
    if (base + i < P.n_bins) P.start[base + i] = sh[pad(i)];
  }
  if (threadIdx.x == 0) P.block_sum[blockIdx.x] = total;
}

// exclusive scan of the tile totals (one block); start[n_bins] = total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_totals(MorseDev P, int n_tiles) {
  const int base = threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = base + i < n_tiles ? P.block_sum[base + i] : 0;
    s += v[i];
  }
  int total;
  int run = block_exclusive(s, total);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n_tiles) P.block_sum[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) P.start[P.n_bins] = total;
}

// add the tile offsets (one thread per bin)
__global__ void k_scan_add(MorseDev P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.n_bins) P.start[i] += P.block_sum[i / SCAN_TILE];
}

__global__ void k_morse_scatter(MorseDev P, MarkersDev m, Box B) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M || P.owner[k] < 0) return;
  const int bin = P.bin_of[k], own = P.owner[k];
  const int slot = P.start[bin] + P.rank[k];
  P.sorted[slot] = make_float4(wrapped_coord(m, B, 0, k), wrapped_coord(m, B, 1, k), wrapped_coord(m, B, 2, k),
                               __int_as_float(own));
  P.sorted_id[slot] = k;
  P.count[bin] = 0;  // counts are not read again this step
  // the first marker claims the bin; a marker of another body marks it mixed
  const int prev = atomicCAS(P.bin_owner + bin, -1, own);
  if (prev != -1 && prev != own) P.bin_owner[bin] = -2;
}

// Neighbour bins along one axis: first .. first + cnt - 1; on periodic axes
// first = b - 1 (-1 at the low end) and indices wrap into [0, nb) (all bins
// when there are fewer than three); on other axes the range is clipped.
struct AxisRange {
  int first, cnt;
};
__device__ __forceinline__ AxisRange axis_range(int b, int nb, bool periodic) {
  AxisRange r;
  if (periodic) {
    if (nb < 3) {
      r.first = 0;
      r.cnt = nb;
    } else {
      r.first = b - 1;
      r.cnt = 3;
    }
  } else {
    r.first = max(b - 1, 0);
    r.cnt = min(b + 1, nb - 1) - r.first + 1;
  }
  return r;
}
__device__ __forceinline__ int range_bin(const AxisRange& r, int d, int nb) {
  const int v = r.first + d;  // in [-1, nb]
  return v < 0 ? v + nb : (v >= nb ? v - nb : v);
}

// Bins around (b0, b1, b2) whose owner is neither `own` nor empty, as a
// 27-bit mask (bit ix + 3 iy + 9 iz); the 27 owner loads are independent.
__device__ __forceinline__ unsigned foreign_bins(const MorseDev& P, const Box& B, int b0, int b1, int b2, int own,
                                                 AxisRange& rx, AxisRange& ry, AxisRange& rz) {
  rx = axis_range(b0, P.nb[0], B.periodic[0] != 0);
  ry = axis_range(b1, P.nb[1], B.periodic[1] != 0);
  rz = axis_range(b2, P.nb[2], B.periodic[2] != 0);
  unsigned mask = 0u;
#pragma unroll
  for (int iz = 0; iz < 3; ++iz)
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      if (iz >= rz.cnt || iy >= ry.cnt) continue;
      const int row = P.nb[0] * (range_bin(ry, iy, P.nb[1]) + P.nb[1] * range_bin(rz, iz, P.nb[2]));
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        if (ix >= rx.cnt) continue;
        const int bo = P.bin_owner[row + range_bin(rx, ix, P.nb[0])];
        if (bo != own && bo != -1) mask |= 1u << (ix + 3 * iy + 9 * iz);
      }
    }
  return mask;
}

__global__ void __launch_bounds__(MORSE_THREADS) k_morse_force(MorseDev P, MarkersDev m, Box B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.start[P.n_bins]) return;
  const float4 p = P.sorted[s];
  const int own = __float_as_int(p.w);
  const int b0 = bin_coord(P, 0, p.x), b1 = bin_coord(P, 1, p.y), b2 = bin_coord(P, 2, p.z);
  AxisRange rx, ry, rz;
  unsigned mask = foreign_bins(P, B, b0, b1, b2, own, rx, ry, rz);
  const float hx = 0.5f * B.n[0], hy = 0.5f * B.n[1], hz = 0.5f * B.n[2];
  float fx = 0.f, fy = 0.f, fz = 0.f;
  while (mask) {
    const int t = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int ix = t % 3, iy = (t / 3) % 3, iz = t / 9;
    const int bin = range_bin(rx, ix, P.nb[0]) +
                    P.nb[0] * (range_bin(ry, iy, P.nb[1]) + P.nb[1] * range_bin(rz, iz, P.nb[2]));
    const int j1 = P.start[bin + 1];
    for (int j = P.start[bin]; j < j1; ++j) {
      const float4 q = P.sorted[j];
      if (__float_as_int(q.w) == own) continue;
      float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
      if (B.periodic[0]) dx = dx > hx ? dx - B.n[0] : (dx < -hx ? dx + B.n[0] : dx);
      if (B.periodic[1]) dy = dy > hy ? dy - B.n[1] : (dy < -hy ? dy + B.n[1] : dy);
      if (B.periodic[2]) dz = dz > hz ? dz - B.n[2] : (dz < -hz ? dz + B.n[2] : dz);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < P.rc2) || r2 == 0.f) continue;
      const float r = sqrtf(r2);
      const float e = expf(-P.alpha * (r - P.r0));
      const float c = 2.0f * P.alpha * P.D0 * (e * e - e) / r;
      fx = fmaf(c, dx, fx);
      fy = fmaf(c, dy, fy);
      fz = fmaf(c, dz, fz);
    }
  }
  const int k = P.sorted_id[s];
  float4 F = m.F[k];
  F.x += fx;
  F.y += fy;
  F.z += fz;
  m.F[k] = F;
}

}  // namespace

int morse_scan_tiles(int n_bins) { return (n_bins + SCAN_TILE - 1) / SCAN_TILE; }
int morse_max_bins() { return SCAN_TILE * SCAN_TILE; }

void launch_morse(const MorseDev& P, const MarkersDev& m, int nx, int ny, int nz, int geometry, cudaStream_t st) {
  if (m.M == 0 || !(P.rc2 > 0.f)) return;
  Box B;
  B.n[0] = nx; B.n[1] = ny; B.n[2] = nz;
  B.periodic[0] = 1;
  B.periodic[1] = geometry == GEOM_PERIODIC;
  B.periodic[2] = geometry != GEOM_TUBE;
  const int grid = (m.M + MORSE_THREADS - 1) / MORSE_THREADS;
  const int tiles = morse_scan_tiles(P.n_bins);
  k_morse_count<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_scan_tiles<<<tiles, SCAN_THREADS, 0, st>>>(P);
  k_scan_totals<<<1, SCAN_THREADS, 0, st>>>(P, tiles);
  k_scan_add<<<(P.n_bins + 255) / 256, 256, 0, st>>>(P);
  k_morse_scatter<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_force<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
}

}  // namespace ibm

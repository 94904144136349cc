// Morse excluded volume between immersed bodies (Eq. morsePotential of
// arXiv:1704.04551, Sec. 2.2):
//   U = D0 (e^{-2 alpha (r - r0)} - 2 e^{-alpha (r - r0)}),  r < rc,
// between markers of different membrane or filament bodies; the force on a
// marker is F = -dU/dr d/r = 2 alpha D0 (e^2 - e) d/r, e = e^{-alpha (r - r0)},
// d its separation from the other marker (nearest image on periodic axes).
//
// A neighbour list with a skin, rebuilt only when needed. Every step a check
// kernel writes each participating marker's wrapped position and raises the
// rebuild flag if a marker has moved more than skin/2 since the last build;
// two markers then cannot have closed in by more than the skin, so every pair
// within rc is in the lists. The rebuild kernels run every step but return
// at once unless the flag is set (no host round trip, graph friendly):
// a cell list with bins at least rc + skin wide (at most 2^26 of them),
// markers counted into bins with atomics, an exclusive prefix sum of the
// counts, markers scattered into bin order (wrapped position and owner body
// packed in a float4), then one thread per sorted marker collects the markers
// of other bodies within rc + skin in the 27 bins around its own. Each bin
// also records whether all its markers belong to one body: a marker first
// loads the owners of its 27 neighbour bins (independent loads, kept as a bit
// mask) and then reads only the bins that hold markers of another body (a
// membrane's own vertices fill most bins around it). The force kernel walks
// the lists. A list longer than its capacity makes the full 27-bin gather
// compute the forces instead, with the cell list rebuilt every step until
// the lists fit again. Positions come from the stencil cache (floor + FP32
// fraction), wrapped into the box on periodic axes, so separations are exact
// to FP32 rounding of a coordinate below the box size.
#include "morse.cuh"
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

// Current wrapped positions for the list walk, and the rebuild test.
__global__ void k_morse_check(MorseDev P, MarkersDev m, Box B) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M) return;
  const int own = P.owner[k];
  if (own < 0) return;
  const size_t M = (size_t)m.M;
  float u[3], w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int c = m.cell[a * M + k];
    const float f = m.frac[a * M + k];
    u[a] = (float)c + f;
    w[a] = (float)(B.periodic[a] ? wrapi(c, B.n[a]) : c) + f;
  }
  P.cur[k] = make_float4(w[0], w[1], w[2], __int_as_float(own));
  const float4 r = P.ref[k];
  const float dx = u[0] - r.x, dy = u[1] - r.y, dz = u[2] - r.z;
  if (dx * dx + dy * dy + dz * dz > P.half_skin2) P.flags[0] = 1;
}

__global__ void k_morse_count(MorseDev P, MarkersDev m, Box B) {
  if (!P.flags[0]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) P.flags[1] = 0;  // set again by the list build if a list overflows
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
  if (!P.flags[0]) return;  // the same for every thread of the block
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
  if (!P.flags[0]) return;  // the same for every thread of the block
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
  if (!P.flags[0]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.n_bins) P.start[i] += P.block_sum[i / SCAN_TILE];
}

__global__ void k_morse_scatter(MorseDev P, MarkersDev m, Box B) {
  if (!P.flags[0]) return;
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

// Periodic image shifts: box lengths on periodic axes, 0 on the others.
struct Images {
  float L[3];
  __device__ explicit Images(const Box& B) {
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = B.periodic[a] ? (float)B.n[a] : 0.f;
  }
};

// Separation p - q with the nearest image on periodic axes.
__device__ __forceinline__ float3 separation(const Images& I, float4 p, float4 q) {
  float d[3] = {p.x - q.x, p.y - q.y, p.z - q.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float L = I.L[a], h = 0.5f * L;
    if (L > 0.f) d[a] = d[a] > h ? d[a] - L : (d[a] < -h ? d[a] + L : d[a]);
  }
  return make_float3(d[0], d[1], d[2]);
}

// Morse constants in registers.
struct MorseConst {
  float rc2, alpha, r0, c2aD;  // c2aD = 2 alpha D0
  __device__ explicit MorseConst(const MorseDev& P) : rc2(P.rc2), alpha(P.alpha), r0(P.r0), c2aD(2.0f * P.alpha * P.D0) {}
};

// Morse force of q on p, added to f (nothing beyond rc or at r = 0).
__device__ __forceinline__ void morse_pair(const MorseConst& K, const Images& I, float4 p, float4 q, float3& f) {
  const float3 d = separation(I, p, q);
  const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
  if (!(r2 < K.rc2) || r2 == 0.f) return;
  const float r = sqrtf(r2);
  const float e = expf(-K.alpha * (r - K.r0));
  const float c = K.c2aD * (e * e - e) / r;
  f.x = fmaf(c, d.x, f.x);
  f.y = fmaf(c, d.y, f.y);
  f.z = fmaf(c, d.z, f.z);
}

// Bin of a sorted marker and the 27 bins around it that hold markers of
// another body.
__device__ __forceinline__ unsigned sorted_neighbourhood(const MorseDev& P, const Box& B, float4 p, AxisRange& rx,
                                                         AxisRange& ry, AxisRange& rz) {
  const int b0 = bin_coord(P, 0, p.x), b1 = bin_coord(P, 1, p.y), b2 = bin_coord(P, 2, p.z);
  return foreign_bins(P, B, b0, b1, b2, __float_as_int(p.w), rx, ry, rz);
}
__device__ __forceinline__ int mask_bin(const MorseDev& P, unsigned t, const AxisRange& rx, const AxisRange& ry,
                                        const AxisRange& rz) {
  const int ix = t % 3, iy = (t / 3) % 3, iz = t / 9;
  return range_bin(rx, ix, P.nb[0]) + P.nb[0] * (range_bin(ry, iy, P.nb[1]) + P.nb[1] * range_bin(rz, iz, P.nb[2]));
}

// List build (one thread per sorted marker): the markers of other bodies
// within rc + skin, in the order of the cell-list gather, and the position
// the displacement test measures from.
__global__ void __launch_bounds__(MORSE_THREADS) k_morse_build(MorseDev P, MarkersDev m, Box B) {
  if (!P.flags[0]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.start[P.n_bins]) return;
  const float4 p = P.sorted[s];
  const int own = __float_as_int(p.w);
  const int k = P.sorted_id[s];
  AxisRange rx, ry, rz;
  unsigned mask = sorted_neighbourhood(P, B, p, rx, ry, rz);
  const Images I(B);
  const float rl2 = P.rl2;
  const int cap = P.cap;
  int* list = P.nbr + (size_t)k * cap;
  int n = 0;
  while (mask) {
    const int t = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int bin = mask_bin(P, t, rx, ry, rz);
    const int j1 = P.start[bin + 1];
    for (int j = P.start[bin]; j < j1; ++j) {
      const float4 q = P.sorted[j];
      if (__float_as_int(q.w) == own) continue;
      const float3 d = separation(I, p, q);
      if (!(d.x * d.x + d.y * d.y + d.z * d.z < rl2)) continue;
      if (n < cap) list[n] = P.sorted_id[j];
      ++n;
    }
  }
  P.n_nbr[k] = min(n, cap);
  if (n > cap) P.flags[1] = 1;
  const size_t M = (size_t)m.M;
  P.ref[k] = make_float4((float)m.cell[k] + m.frac[k], (float)m.cell[M + k] + m.frac[M + k],
                         (float)m.cell[2 * M + k] + m.frac[2 * M + k], 0.f);
}

// Full gather from the cell list (one thread per sorted marker), used while
// a list has overflowed (the cell list is then rebuilt every step).
__global__ void __launch_bounds__(MORSE_THREADS) k_morse_force(MorseDev P, MarkersDev m, Box B) {
  if (!P.flags[1]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.start[P.n_bins]) return;
  const float4 p = P.sorted[s];
  const int own = __float_as_int(p.w);
  AxisRange rx, ry, rz;
  unsigned mask = sorted_neighbourhood(P, B, p, rx, ry, rz);
  const Images I(B);
  const MorseConst K(P);
  float3 f = make_float3(0.f, 0.f, 0.f);
  while (mask) {
    const int t = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int bin = mask_bin(P, t, rx, ry, rz);
    const int j1 = P.start[bin + 1];
    for (int j = P.start[bin]; j < j1; ++j) {
      const float4 q = P.sorted[j];
      if (__float_as_int(q.w) == own) continue;
      morse_pair(K, I, p, q, f);
    }
  }
  const int k = P.sorted_id[s];
  float4 F = m.F[k];
  F.x += f.x;
  F.y += f.y;
  F.z += f.z;
  m.F[k] = F;
}

// List walk (one thread per marker) with this step's positions.
__global__ void __launch_bounds__(MORSE_THREADS) k_morse_list(MorseDev P, MarkersDev m, Box B) {
  if (P.flags[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M || P.owner[k] < 0) return;
  const int n = P.n_nbr[k];
  if (n == 0) return;
  const float4 p = P.cur[k];
  const int* list = P.nbr + (size_t)k * P.cap;
  const Images I(B);
  const MorseConst K(P);
  float3 f = make_float3(0.f, 0.f, 0.f);
  for (int i = 0; i < n; ++i) morse_pair(K, I, p, P.cur[list[i]], f);
  float4 F = m.F[k];
  F.x += f.x;
  F.y += f.y;
  F.z += f.z;
  m.F[k] = F;
}

// Rebuild next step only if the lists overflowed (the check may add a move).
__global__ void k_morse_reset(MorseDev P) { P.flags[0] = P.flags[1]; }

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
  k_morse_check<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_count<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_scan_tiles<<<tiles, SCAN_THREADS, 0, st>>>(P);
  k_scan_totals<<<1, SCAN_THREADS, 0, st>>>(P, tiles);
  k_scan_add<<<(P.n_bins + 255) / 256, 256, 0, st>>>(P);
  k_morse_scatter<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_build<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_force<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_list<<<grid, MORSE_THREADS, 0, st>>>(P, m, B);
  k_morse_reset<<<1, 1, 0, st>>>(P);
}

}  // namespace ibm

// Lattice-Boltzmann kernels: fused BGK collision + Guo forcing + streaming on
// a single in-place population array (AA access pattern), and the kernels
// that initialise, import, export and check that array.
//
// Method: Sec. 2.1 of arXiv:1704.04551 — Eq. lbm (stream + BGK collide +
// force term), Eq. BGKequilibrium (equilibrium), Eq. rho_u (moments with the
// half-force shift), the Guo term F_i, Eq. viscosity (tau).
//
// AA pattern (one array, each cell reads and writes the same 19 slots):
//   even step: f_i(x) is read from A[x][i]; the post-collision f*_i(x) is
//              written to A[x][opp(i)] (a bounced value carries the
//              moving-wall term already);
//   odd step:  f_i(x) is read from A[x - c_i][opp(i)] (from A[x][i] when
//              x - c_i is solid); f*_i(x) is written to A[x + c_i][i], or,
//              when x + c_i is solid, bounced to A[x][opp(i)].
// After an odd step the array holds f(t+1) in the natural layout.
// Populations are stored as deviations d_i = f_i - w_i (scaled in FP16/BF16)
// and all arithmetic is FP32 in deviation form, which keeps the O(u)
// information of f_i ~ w_i in the significand.
#include "common.cuh"
#include "internal.h"
#include "lbm_cell.cuh"

namespace ibm {


// Fused collide-stream-force kernel: one thread per fluid cell, a 2-D grid
// over (x, fluid row). Row data (offsets of the neighbouring rows, which of
// them are solid) come from the precomputed row table, so a thread does no
// integer division and no geometry arithmetic.
constexpr int COLLIDE_THREADS = 128;
// Resident blocks per SM the register budget is sized for (more blocks,
// more loads in flight; fewer registers): measured best at 256^3 with 10
// (48 registers) for the local even step, 9 (56 registers) for the
// neighbour-addressed odd step in FP32 and 10 for it in the half-precision
// formats. FP32: even 324 -> 316 us, odd 356 -> 331 us against 8 blocks (64
// registers); FP16 even 244 -> 228 us.
template <int S, int ODD>
constexpr int collide_min_blocks() {
  return (S == STORE_F32 && ODD) ? 9 : 10;
}

// The grid is one-dimensional (a row count above 65535 blocks does not fit
// the y dimension): block b covers x chunk b % nxb of row block b / nxb,
// x chunks of a row consecutive.
template <int S, int ODD, int GEOM, bool DENSE, bool IDX32>
__global__ void __launch_bounds__(COLLIDE_THREADS, (collide_min_blocks<S, ODD>())) k_collide(LatticeDev L, const RowInfo* __restrict__ rows,
                                                                int n_rows, int nxb) {
  const int rb = blockIdx.x / nxb, xb = blockIdx.x - rb * nxb;
  const int r = rb * blockDim.y + threadIdx.y;
  const int x = xb * blockDim.x + threadIdx.x;
  if (r >= n_rows || x >= L.nx) return;
  const RowInfo R = rows[r];
  // In the neighbour-addressed (odd) step, rows without solid neighbours
  // (all but a ring of rows along walls) skip the bounce-back tests; a warp
  // lies in one row, so the branch is uniform. (The even step reads and
  // writes its own cell only: a second copy there only cost registers.)
  if constexpr (ODD == 1 && GEOM != GEOM_PERIODIC) {
    if (R.smask == 0) {
      collide_cell<S, ODD, GEOM, DENSE, IDX32, true>(L, R, x);
      return;
    }
  }
  collide_cell<S, ODD, GEOM, DENSE, IDX32>(L, R, x);
}

// Equilibrium initialisation from the moments in uw (ux, uy, uz, rho - 1).
template <int S, int GEOM>
__global__ void k_init_equilibrium(LatticeDev L) {
  using P = Pop<S>;
  using T = typename P::T;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.N) return;
  Cell c;
  T* A = reinterpret_cast<T*>(L.pop);
  const size_t N = (size_t)L.N;
  if (!make_cell<GEOM>(L, idx, c)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) P::st(A + i * N + idx, i, 0.f);
    L.uw[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float4 m = L.uw[idx];
  const float rho = 1.0f + m.w;
  const float usq15 = 1.5f * (m.x * m.x + m.y * m.y + m.z * m.z);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cu = cx(i) * m.x + cy(i) * m.y + cz(i) * m.z;
    P::st(A + i * N + idx, i, wgt(i) * (m.w + rho * (3.0f * cu + 4.5f * cu * cu - usq15)));
  }
}

// Natural-layout populations f_i = w_i + d_i, FP64 [19][N]; ODD_NEXT = the
// array is in the post-even-step layout.
template <int S, int GEOM, bool ODD_NEXT>
__global__ void k_export(LatticeDev L, double* out) {
  using P = Pop<S>;
  using T = typename P::T;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.N) return;
  const T* A = reinterpret_cast<const T*>(L.pop);
  const size_t N = (size_t)L.N;
  Cell c;
  if (!make_cell<GEOM>(L, idx, c)) {
    for (int i = 0; i < Q; ++i) out[i * N + idx] = 0.0;
    return;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float d;
    if (!ODD_NEXT || i == 0) {
      d = P::ld(A + i * N + idx, i);
    } else {
      const bool sol = (GEOM != GEOM_PERIODIC) && nb_solid(c, i, -1);
      d = sol ? P::ld(A + i * N + idx, i) : P::ld(A + opp(i) * N + (idx + nb_off(c, i, -1)), opp(i));
    }
    out[i * N + idx] = wgt_d(i) + (double)d;
  }
}

template <int S>
__global__ void k_import(LatticeDev L, const double* in) {
  using P = Pop<S>;
  using T = typename P::T;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.N) return;
  T* A = reinterpret_cast<T*>(L.pop);
  const size_t N = (size_t)L.N;
#pragma unroll
  for (int i = 0; i < Q; ++i) P::st(A + i * N + idx, i, (float)(in[i * N + idx] - wgt_d(i)));
}

// Moments between the API's FP64 layout (rho [N], u [3][N]) and the
// lattice's (u, rho - 1) float4 array: set_lattice's input before the
// equilibrium initialisation, get_fields' output (solid cells report 0).
__global__ void k_set_moments(LatticeDev L, const double* rho, const double* u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.N) return;
  const size_t N = (size_t)L.N;
  const double r = rho ? rho[i] : 1.0;
  L.uw[i] = make_float4(u ? (float)u[i] : 0.f, u ? (float)u[N + i] : 0.f, u ? (float)u[2 * N + i] : 0.f,
                        (float)(r - 1.0));
}

__global__ void k_get_moments(LatticeDev L, double* rho, double* u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.N) return;
  const size_t N = (size_t)L.N;
  const int t = i / L.nx;
  const bool fl = !solid_yz(L, t % L.ny, t / L.ny);
  const float4 v = L.uw[i];
  if (rho) rho[i] = fl ? 1.0 + (double)v.w : 0.0;
  if (u) {
    u[i] = fl ? (double)v.x : 0.0;
    u[N + i] = fl ? (double)v.y : 0.0;
    u[2 * N + i] = fl ? (double)v.z : 0.0;
  }
}

// FP64 sums of the last collision's moments over fluid cells, max |u|, and
// the finiteness check. out: [0] sum(rho - 1), [1..3] sum rho u, [4] number
// of fluid cells; *umax2_bits: max |u|^2 as float bits (atomicMax on the
// bits orders non-negative floats).
__global__ void __launch_bounds__(256) k_diagnostics(LatticeDev L, const RowInfo* __restrict__ rows, int n_rows,
                                                     double* out, unsigned* umax2_bits) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  float m2 = 0.f;
  bool bad = false;
  const long long n = (long long)n_rows * L.nx;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / L.nx);
    const int idx = rows[r].base + (int)(t - (long long)r * L.nx);
    const float4 m = L.uw[idx];
    const double rho = 1.0 + (double)m.w;
    s0 += (double)m.w;
    s1 += rho * m.x; s2 += rho * m.y; s3 += rho * m.z;
    s4 += 1.0;
    m2 = fmaxf(m2, m.x * m.x + m.y * m.y + m.z * m.z);
    bad = bad || !(isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && isfinite(m.w));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    s4 += __shfl_xor_sync(0xffffffffu, s4, o);
    m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  __shared__ double sh[8][5];
  __shared__ float shm[8];
  __shared__ int shbad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) shbad = 0;
  __syncthreads();
  if (lane == 0) {
    sh[warp][0] = s0; sh[warp][1] = s1; sh[warp][2] = s2; sh[warp][3] = s3; sh[warp][4] = s4;
    shm[warp] = m2;
    if (bad) shbad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    float mm = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a0 += sh[w][0]; a1 += sh[w][1]; a2 += sh[w][2]; a3 += sh[w][3]; a4 += sh[w][4];
      mm = fmaxf(mm, shm[w]);
    }
    atomicAdd(out + 0, a0);
    atomicAdd(out + 1, a1);
    atomicAdd(out + 2, a2);
    atomicAdd(out + 3, a3);
    atomicAdd(out + 4, a4);
    if (shbad) {
      atomicExch(L.status, 1);
      atomicMax(umax2_bits, 0x7f800000u);  // +inf
    } else {
      atomicMax(umax2_bits, __float_as_uint(mm));
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {
inline unsigned blocks_for(int n) { return (unsigned)((n + 255) / 256); }

template <int S, int GEOM>
void launch_collide_g(const LatticeDev& L, const RowInfo* rows, int n_rows, bool odd, bool dense, cudaStream_t st) {
  const int tx = L.nx >= COLLIDE_THREADS ? COLLIDE_THREADS : ((L.nx + 31) / 32) * 32;
  const int ty = COLLIDE_THREADS / tx;
  const int nxb = (L.nx + tx - 1) / tx;
  const dim3 block(tx, ty), grid((unsigned)nxb * (unsigned)((n_rows + ty - 1) / ty));
  // 32-bit element offsets in the odd step while 19 N < 2^32 (a build with
  // IBM_FORCE_IDX64 defined always takes the 64-bit variant, so that the
  // parity tests reach it on small lattices)
#ifdef IBM_FORCE_IDX64
  const bool idx32 = false;
#else
  const bool idx32 = (unsigned long long)Q * (unsigned long long)L.N < (1ull << 32);
#endif
  if (odd && idx32) {
    if (dense) k_collide<S, 1, GEOM, true, true><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
    else k_collide<S, 1, GEOM, false, true><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
  } else if (odd) {
    if (dense) k_collide<S, 1, GEOM, true, false><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
    else k_collide<S, 1, GEOM, false, false><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
  } else {
    if (dense) k_collide<S, 0, GEOM, true, false><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
    else k_collide<S, 0, GEOM, false, false><<<grid, block, 0, st>>>(L, rows, n_rows, nxb);
  }
}
template <int S>
void launch_collide_s(const LatticeDev& L, const RowInfo* rows, int n_rows, bool odd, bool dense, cudaStream_t st) {
  switch (L.geometry) {
    case GEOM_PERIODIC: launch_collide_g<S, GEOM_PERIODIC>(L, rows, n_rows, odd, dense, st); break;
    case GEOM_YWALLS: launch_collide_g<S, GEOM_YWALLS>(L, rows, n_rows, odd, dense, st); break;
    default: launch_collide_g<S, GEOM_TUBE>(L, rows, n_rows, odd, dense, st); break;
  }
}
template <int S, int GEOM>
void launch_init_g(const LatticeDev& L, cudaStream_t st) {
  k_init_equilibrium<S, GEOM><<<blocks_for(L.N), 256, 0, st>>>(L);
}
template <int S>
void launch_init_s(const LatticeDev& L, cudaStream_t st) {
  switch (L.geometry) {
    case GEOM_PERIODIC: launch_init_g<S, GEOM_PERIODIC>(L, st); break;
    case GEOM_YWALLS: launch_init_g<S, GEOM_YWALLS>(L, st); break;
    default: launch_init_g<S, GEOM_TUBE>(L, st); break;
  }
}
template <int S, int GEOM>
void launch_export_g(const LatticeDev& L, bool odd_next, double* out, cudaStream_t st) {
  if (odd_next) k_export<S, GEOM, true><<<blocks_for(L.N), 256, 0, st>>>(L, out);
  else k_export<S, GEOM, false><<<blocks_for(L.N), 256, 0, st>>>(L, out);
}
template <int S>
void launch_export_s(const LatticeDev& L, bool odd_next, double* out, cudaStream_t st) {
  switch (L.geometry) {
    case GEOM_PERIODIC: launch_export_g<S, GEOM_PERIODIC>(L, odd_next, out, st); break;
    case GEOM_YWALLS: launch_export_g<S, GEOM_YWALLS>(L, odd_next, out, st); break;
    default: launch_export_g<S, GEOM_TUBE>(L, odd_next, out, st); break;
  }
}
}  // namespace

void launch_collide(const LatticeDev& L, const RowInfo* rows, int n_rows, int storage, bool odd, bool dense,
                    cudaStream_t st) {
  if (n_rows == 0) return;
  switch (storage) {
    case STORE_F32: launch_collide_s<STORE_F32>(L, rows, n_rows, odd, dense, st); break;
    case STORE_F16: launch_collide_s<STORE_F16>(L, rows, n_rows, odd, dense, st); break;
    default: launch_collide_s<STORE_BF16>(L, rows, n_rows, odd, dense, st); break;
  }
}

void launch_init_equilibrium(const LatticeDev& L, int storage, cudaStream_t st) {
  switch (storage) {
    case STORE_F32: launch_init_s<STORE_F32>(L, st); break;
    case STORE_F16: launch_init_s<STORE_F16>(L, st); break;
    default: launch_init_s<STORE_BF16>(L, st); break;
  }
}

void launch_export(const LatticeDev& L, int storage, bool odd_next, double* out, cudaStream_t st) {
  switch (storage) {
    case STORE_F32: launch_export_s<STORE_F32>(L, odd_next, out, st); break;
    case STORE_F16: launch_export_s<STORE_F16>(L, odd_next, out, st); break;
    default: launch_export_s<STORE_BF16>(L, odd_next, out, st); break;
  }
}

void launch_import(const LatticeDev& L, int storage, const double* in, cudaStream_t st) {
  switch (storage) {
    case STORE_F32: k_import<STORE_F32><<<blocks_for(L.N), 256, 0, st>>>(L, in); break;
    case STORE_F16: k_import<STORE_F16><<<blocks_for(L.N), 256, 0, st>>>(L, in); break;
    default: k_import<STORE_BF16><<<blocks_for(L.N), 256, 0, st>>>(L, in); break;
  }
}

void launch_set_moments(const LatticeDev& L, const double* rho, const double* u, cudaStream_t st) {
  k_set_moments<<<blocks_for(L.N), 256, 0, st>>>(L, rho, u);
}

void launch_get_moments(const LatticeDev& L, double* rho, double* u, cudaStream_t st) {
  k_get_moments<<<blocks_for(L.N), 256, 0, st>>>(L, rho, u);
}

void launch_diagnostics(const LatticeDev& L, const RowInfo* rows, int n_rows, double* out, unsigned* umax2_bits,
                        cudaStream_t st) {
  const long long n = (long long)n_rows * L.nx;
  if (n == 0) return;
  const long long blocks = (n + 255) / 256;
  k_diagnostics<<<(unsigned)(blocks < 1216 ? blocks : 1216), 256, 0, st>>>(L, rows, n_rows, out, umax2_bits);
}

}  // namespace ibm

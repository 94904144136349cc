// Device-side bodies of the lattice-Boltzmann kernels, shared by the
// single-lattice kernels (lbm.cu) and the batched serving kernels
// (serve.cu). Method: Sec. 2.1 of arXiv:1704.04551 — Eq. lbm (stream + BGK
// collide + force term), Eq. BGKequilibrium, Eq. rho_u (moments with the
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
#pragma once
#include "common.cuh"

namespace ibm {

namespace lbm_detail {

template <int S>
struct Pop {
  using St = Store<S>;
  using T = typename St::T;
  __device__ static __forceinline__ float ld(const T* p, int i) {
    if constexpr (S == STORE_F32) return *p;
    else if constexpr (S == STORE_F16) return __half2float(*p) * (1.0f / dev_scale(i));
    else return __bfloat162float(*p) * (1.0f / dev_scale(i));
  }
  __device__ static __forceinline__ void st(T* p, int i, float v) {
    if constexpr (S == STORE_F32) *p = v;
    else if constexpr (S == STORE_F16) *p = __float2half_rn(v * dev_scale(i));
    else *p = __float2bfloat16_rn(v * dev_scale(i));
  }
  // the stored value itself (K_i d_i for the half-precision formats)
  __device__ static __forceinline__ float ld_raw(const T* p) {
    if constexpr (S == STORE_F32) return *p;
    else if constexpr (S == STORE_F16) return __half2float(*p);
    else return __bfloat162float(*p);
  }
  __device__ static __forceinline__ void st_raw(T* p, float v) {
    if constexpr (S == STORE_F32) *p = v;
    else if constexpr (S == STORE_F16) *p = __float2half_rn(v);
    else *p = __float2bfloat16_rn(v);
  }
};

struct Cell {
  int x, y, z;
  unsigned smask;          // bit (cy+1)*3 + (cz+1): neighbour in that (y,z) direction is solid
  int oxp, oxm, oyp, oym, ozp, ozm;  // wrapped element offsets of the six axis neighbours
};

template <int GEOM>
__device__ __forceinline__ bool make_cell(const LatticeDev& L, int idx, Cell& c) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  c.x = idx % nx;
  const int t = idx / nx;
  c.y = t % ny;
  c.z = t / ny;
  c.smask = 0u;
  if constexpr (GEOM != GEOM_PERIODIC) {
    if (solid_yz(L, c.y, c.z)) return false;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
        if (solid_yz(L, c.y + dy, c.z + dz)) c.smask |= 1u << ((dy + 1) * 3 + (dz + 1));
  }
  c.oxp = (c.x == nx - 1) ? -(nx - 1) : 1;
  c.oxm = (c.x == 0) ? (nx - 1) : -1;
  const int sy = nx, sz = nx * ny;
  c.oyp = (c.y == ny - 1) ? -(ny - 1) * sy : sy;
  c.oym = (c.y == 0) ? (ny - 1) * sy : -sy;
  c.ozp = (c.z == nz - 1) ? -(nz - 1) * sz : sz;
  c.ozm = (c.z == 0) ? (nz - 1) * sz : -sz;
  return true;
}

// element offset of the neighbour x + s*c_i
__device__ __forceinline__ int nb_off(const Cell& c, int i, int s) {
  const int dx = s * cx(i), dy = s * cy(i), dz = s * cz(i);
  return (dx > 0 ? c.oxp : (dx < 0 ? c.oxm : 0)) + (dy > 0 ? c.oyp : (dy < 0 ? c.oym : 0)) +
         (dz > 0 ? c.ozp : (dz < 0 ? c.ozm : 0));
}
// is x + s*c_i solid?
__device__ __forceinline__ bool nb_solid(const Cell& c, int i, int s) {
  return (c.smask >> ((s * cy(i) + 1) * 3 + (s * cz(i) + 1))) & 1u;
}

}  // namespace lbm_detail
using namespace lbm_detail;

// Collision of one cell (Eqs. rho_u, BGKequilibrium, the Guo term) on its
// 19 loaded values d (in place; the stored values K_i d_i for the
// half-precision formats): moments with the half-force shift (the force
// density is read where the cell's tile is touched, and the moments are
// written there or everywhere with DENSE), BGK relaxation and the Guo term.
// Returns rho (for the moving-wall term of the streaming).
template <int S, bool DENSE>
__device__ __forceinline__ float relax_cell(const LatticeDev& L, float d[Q], int idx, int tile) {
  // HALF: d[] holds the stored values K_i d_i of the half-precision formats
  // (K_i = dev_scale(i), a power of two, so that folding 1/K_i into the
  // moment sums and K_i into the update constants is exact).
  constexpr bool HALF = S != STORE_F32;
  // moments (Eq. rho_u): rho = sum f, rho u = sum f c + g/2
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float k = HALF ? 1.0f / dev_scale(i) : 1.0f;
    drho = fmaf(d[i], k, drho);
    if (cx(i)) jx = fmaf(d[i], cx(i) * k, jx);
    if (cy(i)) jy = fmaf(d[i], cy(i) * k, jy);
    if (cz(i)) jz = fmaf(d[i], cz(i) * k, jz);
  }
  float Gx = L.g0x, Gy = L.g0y, Gz = L.g0z;
  const bool touched = L.flags[tile] != 0;
  if (touched) {
    const float4 gg = L.g[idx];
    Gx += gg.x; Gy += gg.y; Gz += gg.z;
  }
  const float rho = 1.0f + drho;
  const float irho = 1.0f / rho;
  const float ux = (jx + 0.5f * Gx) * irho;
  const float uy = (jy + 0.5f * Gy) * irho;
  const float uz = (jz + 0.5f * Gz) * irho;
  if (DENSE || touched) L.uw[idx] = make_float4(ux, uy, uz, drho);

  // BGK relaxation toward the equilibrium (Eq. BGKequilibrium) plus the Guo
  // term. Written per direction: a form that shares the parts of opposite
  // directions (c_{i+1} = -c_i) saves a few percent of the collide time but
  // doubled the FP32 velocity error against the FP64 oracle after 1000
  // coupled steps of the red-cell tube (1.8e-5 vs 9.4e-6, measured).
  const float om = L.omega, pre = L.guo_pre;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float uG = ux * Gx + uy * Gy + uz * Gz;
  if constexpr (!HALF) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float w = wgt(i);
      const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
      const float cG = cx(i) * Gx + cy(i) * Gy + cz(i) * Gz;
      const float deq = w * (drho + rho * (3.0f * cu + 4.5f * cu * cu - usq15));
      const float Fi = pre * w * (3.0f * (cG - uG) + 9.0f * cu * cG);
      d[i] = d[i] + om * (deq - d[i]) + Fi;
    }
  } else {
    // The same update, regrouped for the half-precision formats (their
    // rounding dominates the error): with cu = c.u and cG = c.G,
    //   K_i (om f^eq_i + F_i) = K_i w_i [T0 + cu (3 om rho + 4.5 om rho cu + 9 pre cG) + 3 pre cG],
    //   T0 = om (drho - rho 1.5 u^2) - 3 pre u.G,
    // K_i w_i = 8/9 for every moving direction (4/3 at rest), and the pair
    // i, i+1 = opp(i) shares the even part in cu and flips the odd part.
    const float om1 = 1.0f - om;
    const float T0 = om * (drho - rho * usq15) - 3.0f * pre * uG;
    constexpr float KW = 8.0f / 9.0f;
    const float A = (KW * 3.0f) * om * rho, B = (KW * 4.5f) * om * rho;
    const float P3 = (KW * 3.0f) * pre, P9 = (KW * 9.0f) * pre;
    const float T0w = KW * T0;
    d[0] = fmaf(om1, d[0], (4.0f / 3.0f) * T0);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
      const float cG = cx(i) * Gx + cy(i) * Gy + cz(i) * Gz;
      const float even = fmaf(fmaf(B, cu, P9 * cG), cu, T0w);
      const float odd = fmaf(A, cu, P3 * cG);
      d[i] = fmaf(om1, d[i], even + odd);
      d[i + 1] = fmaf(om1, d[i + 1], even - odd);
    }
  }

  return rho;
}

// One fluid cell of the fused collide-stream-force step (x in the row R).
// IDX32: element offsets of the neighbour-addressed (odd) step computed in
// 32 bits, valid while 19 N < 2^32 (fewer integer instructions than 64-bit
// address arithmetic per population; the odd step is issue-bound).
// INTERIOR: the row's y/z neighbour rows are all fluid (R.smask == 0), so
// no population is bounced back and the solid tests drop out.
template <int S, int ODD, int GEOM, bool DENSE, bool IDX32 = false, bool INTERIOR = false>
__device__ __forceinline__ void collide_cell(const LatticeDev& L, const RowInfo& R, int x) {
  constexpr bool WALLS = GEOM != GEOM_PERIODIC && !INTERIOR;  // solid neighbours possible
  using P = Pop<S>;
  using T = typename P::T;
  const int idx = R.base + x;
  Cell c;
  c.x = x;
  c.y = R.y;
  c.smask = (unsigned)R.smask;
  c.oxp = (x == L.nx - 1) ? 1 - L.nx : 1;
  c.oxm = (x == 0) ? L.nx - 1 : -1;
  c.oyp = R.oyp; c.oym = R.oym; c.ozp = R.ozp; c.ozm = R.ozm;
  T* A = reinterpret_cast<T*>(L.pop);
  const size_t N = (size_t)L.N;

  // f_j(x) sits at A[x][j] (even step) or at A[x - c_j][opp(j)] (odd step;
  // A[x][j] if x - c_j is solid). In both parities f*_i(x) goes back to the
  // slot that held f_opp(i)(x), which covers streaming and half-way
  // bounce-back alike.
  // element offset of population j at cell e (32- or 64-bit arithmetic)
  auto elem = [&](int j, int e) -> const T* {
    if constexpr (IDX32) return A + (unsigned)((unsigned)j * (unsigned)N + (unsigned)e);
    else return A + (size_t)j * N + e;
  };
  constexpr bool HALF = S != STORE_F32;  // d[] holds K_i d_i (see relax_cell)
  float d[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    if (!ODD || j == 0 || (WALLS && nb_solid(c, j, -1)))
      d[j] = P::ld_raw(elem(j, idx));
    else
      d[j] = P::ld_raw(elem(opp(j), idx + nb_off(c, j, -1)));
  }

  const float rho = relax_cell<S, DENSE>(L, d, idx, R.trow + (x >> TILE_X_SHIFT));

  // Recompute the write addresses from a few laundered registers instead of
  // keeping the 19 read addresses alive across the collision (which spills).
  int widx = idx;
  asm volatile("" : "+r"(widx), "+r"(c.oxp), "+r"(c.oxm), "+r"(c.oyp), "+r"(c.oym), "+r"(c.ozp), "+r"(c.ozm),
               "+r"(c.smask));
  // streaming with half-way bounce-back (moving-wall term on y walls)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float v = d[i];
    const bool sol = WALLS && i != 0 && nb_solid(c, i, +1);
    if (GEOM == GEOM_YWALLS && sol && cx(i) != 0) {
      // stored into slot opp(i): the half-precision scale of that slot
      const float uw = (c.y + cy(i) < 0) ? L.wall_u0 : L.wall_u1;
      v -= (HALF ? dev_scale(opp(i)) : 1.0f) * 6.0f * wgt(i) * rho * (float)cx(i) * uw;
    }
    if (!ODD || i == 0 || sol)
      P::st_raw(const_cast<T*>(elem(opp(i), widx)), v);
    else
      P::st_raw(const_cast<T*>(elem(i, widx + nb_off(c, i, +1))), v);
  }
}


}  // namespace ibm

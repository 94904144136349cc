// Immersed-boundary transfer kernels (Sec. 2.3 of arXiv:1704.04551):
//   spread       g(x) += F_k delta(x - X_k)          (Eq. ibmForceSpread)
//   interpolate  U_k = sum_x u(x) delta(x - X_k),    (Eq. ibmVelocityInterpret)
//                then X_k += U_k (explicit advection, dt = 1)
// with delta(x) = phi(x) phi(y) phi(z), phi(r) = (1 + cos(pi r / 2)) / 4 for
// |r| <= 2 (Eq. deltaPhiSimple). The 4-point stencil of a marker at X is the
// nodes floor(X)-1 .. floor(X)+2 on each axis; nodes inside walls or the
// tube's solid are skipped (no renormalisation). Periodic axes wrap.
#include "common.cuh"
#include "internal.h"

namespace ibm {

namespace {

struct Stencil {
  int bx, by, bz;        // first node on each axis (unwrapped)
  float wx[4], wy[4], wz[4];
};

// Marker position (FP64) -> stencil base and FP32 weights. The fractional
// offset s = X - floor(X) is formed in FP64 and rounded once to FP32.
__device__ __forceinline__ void make_stencil(double X, double Y, double Z, Stencil& s) {
  const double fx = floor(X), fy = floor(Y), fz = floor(Z);
  s.bx = (int)fx - 1; s.by = (int)fy - 1; s.bz = (int)fz - 1;
  const float ox = (float)(X - fx), oy = (float)(Y - fy), oz = (float)(Z - fz);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // node b + k sits at distance r = (k - 1) - offset from X
    s.wx[k] = 0.25f * (1.0f + cospif(0.5f * ((float)(k - 1) - ox)));
    s.wy[k] = 0.25f * (1.0f + cospif(0.5f * ((float)(k - 1) - oy)));
    s.wz[k] = 0.25f * (1.0f + cospif(0.5f * ((float)(k - 1) - oz)));
  }
}

}  // namespace

template <int GEOM>
__global__ void __launch_bounds__(256) k_spread(LatticeDev L, MarkersDev m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M) return;
  const size_t M = (size_t)m.M;
  Stencil s;
  make_stencil(m.X[k], m.X[M + k], m.X[2 * M + k], s);
  const float4 F = m.F[k];
  int xs[4], tx[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    xs[a] = wrapi(s.bx + a, L.nx);
    tx[a] = xs[a] >> TILE_X_SHIFT;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int z = s.bz + c;
    if (GEOM != GEOM_TUBE) z = wrapi(z, L.nz);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int y = s.by + b;
      if (GEOM == GEOM_PERIODIC) y = wrapi(y, L.ny);
      if (GEOM != GEOM_PERIODIC && solid_yz(L, y, z)) continue;
      const float wyz = s.wy[b] * s.wz[c];
      const int row = L.nx * (y + L.ny * z);
      const int trow = L.ntx * ((y >> TILE_Y_SHIFT) + L.nty * (z >> TILE_Z_SHIFT));
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = s.wx[a] * wyz;
        atomicAdd(L.g + row + xs[a], make_float4(F.x * w, F.y * w, F.z * w, 0.f));
        if (a == 0 || tx[a] != tx[a - 1]) L.flags[trow + tx[a]] = 1;
      }
    }
  }
}

template <int GEOM>
__global__ void __launch_bounds__(256) k_interpolate(LatticeDev L, MarkersDev m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M) return;
  const size_t M = (size_t)m.M;
  const double X = m.X[k], Y = m.X[M + k], Z = m.X[2 * M + k];
  Stencil s;
  make_stencil(X, Y, Z, s);
  int xs[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) xs[a] = wrapi(s.bx + a, L.nx);
  float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int z = s.bz + c;
    if (GEOM != GEOM_TUBE) z = wrapi(z, L.nz);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int y = s.by + b;
      if (GEOM == GEOM_PERIODIC) y = wrapi(y, L.ny);
      if (GEOM != GEOM_PERIODIC && solid_yz(L, y, z)) continue;
      const float wyz = s.wy[b] * s.wz[c];
      const float4* row = L.uw + L.nx * (y + L.ny * z);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = s.wx[a] * wyz;
        const float4 u = row[xs[a]];
        ux = fmaf(w, u.x, ux);
        uy = fmaf(w, u.y, uy);
        uz = fmaf(w, u.z, uz);
      }
    }
  }
  m.U[k] = make_float4(ux, uy, uz, 0.f);
  m.X[k] = X + (double)ux;
  m.X[M + k] = Y + (double)uy;
  m.X[2 * M + k] = Z + (double)uz;
}

void launch_spread(const LatticeDev& L, const MarkersDev& m, cudaStream_t st) {
  if (m.M == 0) return;
  const unsigned nb = (unsigned)((m.M + 255) / 256);
  switch (L.geometry) {
    case GEOM_PERIODIC: k_spread<GEOM_PERIODIC><<<nb, 256, 0, st>>>(L, m); break;
    case GEOM_YWALLS: k_spread<GEOM_YWALLS><<<nb, 256, 0, st>>>(L, m); break;
    default: k_spread<GEOM_TUBE><<<nb, 256, 0, st>>>(L, m); break;
  }
}

void launch_interpolate(const LatticeDev& L, const MarkersDev& m, cudaStream_t st) {
  if (m.M == 0) return;
  const unsigned nb = (unsigned)((m.M + 255) / 256);
  switch (L.geometry) {
    case GEOM_PERIODIC: k_interpolate<GEOM_PERIODIC><<<nb, 256, 0, st>>>(L, m); break;
    case GEOM_YWALLS: k_interpolate<GEOM_YWALLS><<<nb, 256, 0, st>>>(L, m); break;
    default: k_interpolate<GEOM_TUBE><<<nb, 256, 0, st>>>(L, m); break;
  }
}

}  // namespace ibm

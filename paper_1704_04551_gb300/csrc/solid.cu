// Solid-only dynamics of the markers (the membrane stretching validation of
// Sec. 3.2 of arXiv:1704.04551): velocity Verlet with viscous damping under
// the bodies' own forces, the Morse term and an external force, no fluid.
//   first half:  v' = v + dt/2 (F(X)/m - gamma v);  X += dt v'
//   second half: v  = (v' + dt/2 F(X)/m) / (1 + gamma dt/2)
// One thread per marker coordinate; positions stay FP64 and the stencil
// cache is refreshed after each move.
#include "common.cuh"
#include "internal.h"

namespace ibm {

namespace {

__device__ __forceinline__ float force_comp(const MarkersDev& m, int a, int k) {
  const float4 F = m.F[k];
  return a == 0 ? F.x : (a == 1 ? F.y : F.z);
}

__global__ void k_solid_first(MarkersDev m, double* v, const double* fext, double dt, double gamma, double mass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * m.M) return;
  const int a = i / m.M, k = i - a * m.M;
  const double F = (double)force_comp(m, a, k) + (fext ? fext[i] : 0.0);
  const double vh = v[i] + 0.5 * dt * (F / mass - gamma * v[i]);
  v[i] = vh;
  const double X = m.X[i] + dt * vh;
  m.X[i] = X;
  cache_coord(m, i, X);
}

__global__ void k_solid_second(MarkersDev m, double* v, const double* fext, double dt, double gamma, double mass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * m.M) return;
  const int a = i / m.M, k = i - a * m.M;
  const double F = (double)force_comp(m, a, k) + (fext ? fext[i] : 0.0);
  v[i] = (v[i] + 0.5 * dt * F / mass) / (1.0 + 0.5 * gamma * dt);
}

}  // namespace

void launch_solid_half(const MarkersDev& m, double* v, const double* fext, double dt, double gamma, double mass,
                       bool first, cudaStream_t st) {
  if (m.M == 0) return;
  const int n = 3 * m.M;
  if (first) k_solid_first<<<(n + 255) / 256, 256, 0, st>>>(m, v, fext, dt, gamma, mass);
  else k_solid_second<<<(n + 255) / 256, 256, 0, st>>>(m, v, fext, dt, gamma, mass);
}

}  // namespace ibm

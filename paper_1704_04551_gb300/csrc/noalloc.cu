// Force spreading without device allocation (ibm_lbm_spread_noalloc).
//
// For callers that cannot call cudaMalloc (a framework that has reserved the
// GPU's memory for its own pool, a loop that may not pay allocation cost):
// the accumulator lives in a file-scope device array of fixed size instead
// of memory the library allocates. The operation is the spreading of Eq.
// ibmForceSpread with the 4-point cosine delta of Eq. deltaPhiSimple, the
// same as the SPREAD stage of a handle.
#include <cuda_runtime.h>

#include "../../include/ibm_lbm.h"
#include "common.cuh"

namespace ibm {
namespace {

// One accumulator per device, shared by every call on that device. In host
// code this name is only a stand-in for the device array; its device address
// comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float4 g_noalloc_scratch[IBM_LBM_NOALLOC_MAX_CELLS];

// Device address of the accumulator in the current context. Looked up on
// every call (a host-side table lookup once the module is loaded) rather than
// cached: if the caller resets the device, the module is loaded again and the
// array may move, and a cached address would then point at freed memory.
cudaError_t scratch_address(float4** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<float4*>(p);
  return cudaSuccess;
}

struct Grid {
  int nx, ny, nz, N, geometry;
  float yc, zc, R2;
};

__device__ __forceinline__ bool grid_solid(const Grid& G, int y, int z) {
  if (G.geometry == GEOM_YWALLS) return (unsigned)y >= (unsigned)G.ny;
  if (G.geometry == GEOM_TUBE) {
    if ((unsigned)y >= (unsigned)G.ny || (unsigned)z >= (unsigned)G.nz) return true;
    const float dy = (float)y - G.yc, dz = (float)z - G.zc;
    return dy * dy + dz * dz > G.R2;
  }
  return false;
}

__global__ void k_spread_noalloc(Grid G, const double* __restrict__ X, const double* __restrict__ F, int M,
                                 float4* acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const double px = X[k], py = X[(size_t)M + k], pz = X[2 * (size_t)M + k];
  // Positions come straight from device memory, unchecked by the host: a
  // marker that is not finite or lies at |x| >= 2^30 (the bound the handle's
  // set_markers enforces) is skipped, so that no index below overflows.
  const double lim = 1073741824.0;
  if (!(fabs(px) < lim && fabs(py) < lim && fabs(pz) < lim)) return;
  const float fx = (float)F[k], fy = (float)F[(size_t)M + k], fz = (float)F[2 * (size_t)M + k];
  const double bx = floor(px), by = floor(py), bz = floor(pz);
  const float ox = (float)(px - bx), oy = (float)(py - by), oz = (float)(pz - bz);
  float wx[4], wy[4], wz[4];
  int xs[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    wx[a] = 0.25f * (1.0f + cospif(0.5f * ((float)(a - 1) - ox)));
    wy[a] = 0.25f * (1.0f + cospif(0.5f * ((float)(a - 1) - oy)));
    wz[a] = 0.25f * (1.0f + cospif(0.5f * ((float)(a - 1) - oz)));
    xs[a] = wrapi((int)bx - 1 + a, G.nx);
  }
  for (int c = 0; c < 4; ++c) {
    int z = (int)bz - 1 + c;
    if (G.geometry != GEOM_TUBE) z = wrapi(z, G.nz);
    for (int b = 0; b < 4; ++b) {
      int y = (int)by - 1 + b;
      if (G.geometry == GEOM_PERIODIC) y = wrapi(y, G.ny);
      if (grid_solid(G, y, z)) continue;
      const float wyz = wy[b] * wz[c];
      float4* row = acc + G.nx * (y + G.ny * z);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = wx[a] * wyz;
        atomicAdd(row + xs[a], make_float4(fx * w, fy * w, fz * w, 0.f));
      }
    }
  }
}

__global__ void k_scatter_noalloc(const float4* acc, int N, double* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 v = acc[i];
  g[i] = v.x;
  g[(size_t)N + i] = v.y;
  g[2 * (size_t)N + i] = v.z;
}

}  // namespace
}  // namespace ibm

namespace {
int spread_noalloc(const double* X, const double* F, int64_t n_markers, int32_t nx, int32_t ny, int32_t nz,
                   int32_t geometry, double tube_radius, double* g, void* stream) {
  using namespace ibm;
  const long long N = (long long)nx * ny * nz;
  if (nx < 4 || ny < 4 || nz < 4 || N > IBM_LBM_NOALLOC_MAX_CELLS) return IBM_LBM_E_ARG;
  if (n_markers < 0 || n_markers >= (1LL << 31) || (n_markers > 0 && (!X || !F)) || !g) return IBM_LBM_E_ARG;
  if (geometry < 0 || geometry > 2 || (geometry == 2 && !(tube_radius > 0))) return IBM_LBM_E_ARG;
  float4* acc = nullptr;
  if (scratch_address(&acc) != cudaSuccess) {
    cudaGetLastError();
    return IBM_LBM_E_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Grid G{nx, ny, nz, (int)N, geometry, 0.5f * (float)(ny - 1), 0.5f * (float)(nz - 1),
         (float)(tube_radius * tube_radius)};
  if (cudaMemsetAsync(acc, 0, sizeof(float4) * (size_t)N, st) != cudaSuccess) {
    cudaGetLastError();
    return IBM_LBM_E_CUDA;
  }
  const int M = (int)n_markers;
  if (M > 0) k_spread_noalloc<<<(M + 255) / 256, 256, 0, st>>>(G, X, F, M, acc);
  k_scatter_noalloc<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(acc, (int)N, g);
  if (cudaGetLastError() != cudaSuccess) return IBM_LBM_E_CUDA;
  return IBM_LBM_OK;
}
}  // namespace

// No C++ exception crosses the C ABI (there is no handle to carry a message).
extern "C" int ibm_lbm_spread_noalloc(const double* X, const double* F, int64_t n_markers, int32_t nx, int32_t ny,
                                      int32_t nz, int32_t geometry, double tube_radius, double* g,
                                      void* stream) {
  try {
    return spread_noalloc(X, F, n_markers, nx, ny, nz, geometry, tube_radius, g, stream);
  } catch (...) {
    return IBM_LBM_E_ARG;
  }
}

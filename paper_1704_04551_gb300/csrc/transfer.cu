// Immersed-boundary transfer kernels of one lattice (Sec. 2.3 of
// arXiv:1704.04551): spreading (Eq. ibmForceSpread) and interpolation with
// advection (Eq. ibmVelocityInterpret), one thread block per marker group;
// the group bodies and their design notes are in transfer_group.cuh.
#include "common.cuh"
#include "internal.h"
#include "transfer_group.cuh"

namespace ibm {

// Stencil cache from the positions (after set_markers).
__global__ void k_stencil_cache(MarkersDev m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.M) return;
  const size_t M = (size_t)m.M;
  for (int a = 0; a < 3; ++a) cache_coord(m, a * M + k, m.X[a * M + k]);
}

template <int GEOM>
__global__ void __launch_bounds__(XFER_THREADS, 2) k_spread(LatticeDev L, MarkersDev m, const MarkerGroup* groups,
                                                            int4* boxes) {
  extern __shared__ __align__(16) unsigned char smem[];  // fixed-point box, marker records
  spread_group<GEOM>(L, m, groups[blockIdx.x], boxes + 2 * blockIdx.x, smem);
}

template <int GEOM>
__global__ void __launch_bounds__(XFER_THREADS, 2) k_interpolate(LatticeDev L, MarkersDev m,
                                                                 const MarkerGroup* groups, const int4* boxes) {
  extern __shared__ __align__(16) unsigned char smem[];  // velocity box, marker records
  interpolate_group<GEOM>(L, m, groups[blockIdx.x], boxes + 2 * blockIdx.x, smem);
}

// The same for launches of fewer than LANE_MAX_GROUPS groups (four lanes
// per marker).
template <int GEOM>
__global__ void __launch_bounds__(LANE_THREADS, 1) k_spread_lanes(LatticeDev L, MarkersDev m,
                                                                 const MarkerGroup* groups, int4* boxes) {
  extern __shared__ __align__(16) int ibox[];  // fixed-point box
  spread_group_lanes<GEOM>(L, m, groups[blockIdx.x], boxes + 2 * blockIdx.x, ibox);
}

template <int GEOM>
__global__ void __launch_bounds__(LANE_THREADS, 1) k_interpolate_lanes(LatticeDev L, MarkersDev m,
                                                                      const MarkerGroup* groups, const int4* boxes) {
  extern __shared__ __align__(16) unsigned char smem[];  // velocity box
  interpolate_group_lanes<GEOM>(L, m, groups[blockIdx.x], boxes + 2 * blockIdx.x, smem);
}

cudaError_t transfer_configure() {
  cudaError_t e = cudaSuccess;
#define CFG(k, smem) if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
  CFG(k_spread<GEOM_PERIODIC>, SPREAD_SMEM); CFG(k_spread<GEOM_YWALLS>, SPREAD_SMEM); CFG(k_spread<GEOM_TUBE>, SPREAD_SMEM);
  CFG(k_interpolate<GEOM_PERIODIC>, INTERP_SMEM); CFG(k_interpolate<GEOM_YWALLS>, INTERP_SMEM);
  CFG(k_interpolate<GEOM_TUBE>, INTERP_SMEM);
  CFG(k_spread_lanes<GEOM_PERIODIC>, SPREAD_LANES_SMEM); CFG(k_spread_lanes<GEOM_YWALLS>, SPREAD_LANES_SMEM);
  CFG(k_spread_lanes<GEOM_TUBE>, SPREAD_LANES_SMEM);
  CFG(k_interpolate_lanes<GEOM_PERIODIC>, INTERP_SMEM); CFG(k_interpolate_lanes<GEOM_YWALLS>, INTERP_SMEM);
  CFG(k_interpolate_lanes<GEOM_TUBE>, INTERP_SMEM);
#undef CFG
  return e;
}

// (x, y, z, -) float4 [M] -> FP64 [3][M] (marker velocities and forces for
// the API).
__global__ void k_expand_xyz(const float4* in, double* out, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const float4 v = in[k];
  out[k] = v.x;
  out[(size_t)M + k] = v.y;
  out[2 * (size_t)M + k] = v.z;
}

void launch_expand_xyz(const float4* in, double* out, int M, cudaStream_t st) {
  if (M > 0) k_expand_xyz<<<(M + 255) / 256, 256, 0, st>>>(in, out, M);
}

void launch_stencil_cache(const MarkersDev& m, cudaStream_t st) {
  if (m.M == 0) return;
  k_stencil_cache<<<(m.M + 255) / 256, 256, 0, st>>>(m);
}

void launch_spread(const LatticeDev& L, const MarkersDev& m, const MarkerGroup* groups, int n_groups, int4* boxes,
                   cudaStream_t st) {
  if (m.M == 0 || n_groups == 0) return;
  if (n_groups < LANE_MAX_GROUPS) {
    const size_t smem = SPREAD_LANES_SMEM;
    switch (L.geometry) {
      case GEOM_PERIODIC: k_spread_lanes<GEOM_PERIODIC><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes); break;
      case GEOM_YWALLS: k_spread_lanes<GEOM_YWALLS><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes); break;
      default: k_spread_lanes<GEOM_TUBE><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes); break;
    }
    return;
  }
  const size_t smem = SPREAD_SMEM;
  switch (L.geometry) {
    case GEOM_PERIODIC: k_spread<GEOM_PERIODIC><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
    case GEOM_YWALLS: k_spread<GEOM_YWALLS><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
    default: k_spread<GEOM_TUBE><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
  }
}

void launch_interpolate(const LatticeDev& L, const MarkersDev& m, const MarkerGroup* groups, int n_groups,
                        const int4* boxes, cudaStream_t st) {
  if (m.M == 0 || n_groups == 0) return;
  const size_t smem = INTERP_SMEM;
  if (n_groups < LANE_MAX_GROUPS) {
    switch (L.geometry) {
      case GEOM_PERIODIC:
        k_interpolate_lanes<GEOM_PERIODIC><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes);
        break;
      case GEOM_YWALLS: k_interpolate_lanes<GEOM_YWALLS><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes); break;
      default: k_interpolate_lanes<GEOM_TUBE><<<n_groups, LANE_THREADS, smem, st>>>(L, m, groups, boxes); break;
    }
    return;
  }
  switch (L.geometry) {
    case GEOM_PERIODIC: k_interpolate<GEOM_PERIODIC><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
    case GEOM_YWALLS: k_interpolate<GEOM_YWALLS><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
    default: k_interpolate<GEOM_TUBE><<<n_groups, XFER_THREADS, smem, st>>>(L, m, groups, boxes); break;
  }
}

}  // namespace ibm

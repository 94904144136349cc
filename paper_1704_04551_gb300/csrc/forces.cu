// Marker-force kernels of one lattice: membranes and filaments (Sec. 2.2)
// and rigid bodies (Sec. 2.3), one block per body; the bodies and their
// design notes are in forces_body.cuh.
#include "common.cuh"
#include "forces_body.cuh"
#include "internal.h"

namespace ibm {

__global__ void __launch_bounds__(MEMBRANE_THREADS, 4)
    k_membranes(MarkersDev m, BodyDev* __restrict__ bodies, const int* __restrict__ list, MeshDev mesh) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * 32];
  membrane_block(m, bodies + list[blockIdx.x], mesh, smem, red);
}

__global__ void __launch_bounds__(RIGID_THREADS) k_rigid(MarkersDev m, BodyDev* __restrict__ bodies,
                                                         const int* __restrict__ list) {
  __shared__ double sh[6 * 32];
  rigid_block(m, bodies + list[blockIdx.x], sh);
}

__global__ void __launch_bounds__(FILAMENT_THREADS) k_filaments(MarkersDev m, const BodyDev* __restrict__ bodies,
                                                                 const int* __restrict__ list) {
  filament_block(m, bodies[list[blockIdx.x]]);
}

void launch_filaments(const MarkersDev& m, const BodyDev* bodies, const int* list, int n, cudaStream_t st) {
  if (n > 0) k_filaments<<<n, FILAMENT_THREADS, 0, st>>>(m, bodies, list);
}

size_t membrane_work_floats(int nv, int nt, int ne) {
  (void)ne;
  return (size_t)9 * nv + (size_t)4 * nt;
}

cudaError_t forces_configure(const MeshDev& mesh, size_t max_smem) {
  const size_t work = sizeof(float) * mesh.work_floats;
  if (work + 1024 > max_smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_membranes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work);
}

void launch_forces(const MarkersDev& m, BodyDev* bodies, const int* membranes, int n_membranes, const int* rigids,
                   int n_rigids, const MeshDev& mesh, cudaStream_t st) {
  if (n_rigids > 0) k_rigid<<<n_rigids, RIGID_THREADS, 0, st>>>(m, bodies, rigids);
  if (n_membranes == 0) return;
  k_membranes<<<n_membranes, MEMBRANE_THREADS, sizeof(float) * mesh.work_floats, st>>>(m, bodies, membranes, mesh);
}

}  // namespace ibm

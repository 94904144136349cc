// Internal launchers shared between the kernel files and the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace ibm {

// lbm.cu
void launch_collide(const LatticeDev& L, int storage, bool odd, bool dense, cudaStream_t st);
void launch_init_equilibrium(const LatticeDev& L, int storage, cudaStream_t st);
void launch_export(const LatticeDev& L, int storage, bool odd_next, double* out, cudaStream_t st);
void launch_import(const LatticeDev& L, int storage, const double* in, cudaStream_t st);
void launch_diagnostics(const LatticeDev& L, double* out, unsigned* umax2_bits, cudaStream_t st);

// transfer.cu
void launch_spread(const LatticeDev& L, const MarkersDev& m, cudaStream_t st);
void launch_interpolate(const LatticeDev& L, const MarkersDev& m, cudaStream_t st);

// forces.cu
void launch_forces(const MarkersDev& m, BodyDev* bodies, int n_bodies, const MeshDev& mesh,
                   cudaStream_t st);
size_t forces_smem_bytes(int nv);
cudaError_t forces_configure(size_t smem_bytes);

}  // namespace ibm

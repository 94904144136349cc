// Internal launchers shared between the kernel files and the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "morse.cuh"

namespace ibm {

// lbm.cu
void launch_collide(const LatticeDev& L, const RowInfo* rows, int n_rows, int storage, bool odd, bool dense,
                    cudaStream_t st);
void launch_init_equilibrium(const LatticeDev& L, int storage, cudaStream_t st);
void launch_export(const LatticeDev& L, int storage, bool odd_next, double* out, cudaStream_t st);
void launch_import(const LatticeDev& L, int storage, const double* in, cudaStream_t st);
void launch_set_moments(const LatticeDev& L, const double* rho, const double* u, cudaStream_t st);
void launch_get_moments(const LatticeDev& L, double* rho, double* u, cudaStream_t st);
void launch_diagnostics(const LatticeDev& L, const RowInfo* rows, int n_rows, double* out, unsigned* umax2_bits,
                        cudaStream_t st);

// transfer.cu
void launch_spread(const LatticeDev& L, const MarkersDev& m, const MarkerGroup* groups, int n_groups, int4* boxes,
                   cudaStream_t st);
void launch_interpolate(const LatticeDev& L, const MarkersDev& m, const MarkerGroup* groups, int n_groups,
                        const int4* boxes, cudaStream_t st);
cudaError_t transfer_configure();
void launch_stencil_cache(const MarkersDev& m, cudaStream_t st);
void launch_expand_xyz(const float4* in, double* out, int M, cudaStream_t st);

// forces.cu
void launch_forces(const MarkersDev& m, BodyDev* bodies, const int* membranes, int n_membranes, const int* rigids,
                   int n_rigids, const MeshDev& mesh, cudaStream_t st);
size_t membrane_work_floats(int nv, int nt, int ne);
cudaError_t forces_configure(const MeshDev& mesh, size_t max_smem);
void launch_filaments(const MarkersDev& m, const BodyDev* bodies, const int* list, int n, cudaStream_t st);

// couple.cu (membrane suspensions: interpolation, forces and spreading fused per body)
bool couple_fits(const MeshDev& mesh);
size_t couple_order_bytes(const MeshDev& mesh);
cudaError_t couple_configure();
void launch_couple(const LatticeDev& L, float4* g_next, const MarkersDev& m, BodyDev* bodies, const int2* items,
                   int n_items, const MarkerGroup* groups, int4* boxes, unsigned char* orders, const MeshDev& mesh,
                   cudaStream_t st);

// solid.cu
void launch_solid_half(const MarkersDev& m, double* v, const double* fext, double dt, double gamma, double mass,
                       bool first, cudaStream_t st);

// morse.cu
void launch_morse(const MorseDev& P, const MarkersDev& m, int nx, int ny, int nz, int geometry, cudaStream_t st);
int morse_scan_tiles(int n_bins);
int morse_max_bins();

}  // namespace ibm

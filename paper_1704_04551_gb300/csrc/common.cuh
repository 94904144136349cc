// Device-side definitions shared by the kernels of the coupled IBM-LBM step.
// Lattice: D3Q19 (Sec. 2.1 of arXiv:1704.04551), c_s^2 = 1/3 (Eq. viscosity).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ibm {

constexpr int Q = 19;

// Velocities in the public D3Q19 order: rest, +-x, +-y, +-z, then the face
// diagonals in opposite pairs, so that opposite(i) = i + 1 for odd i and
// i - 1 for even i > 0.
__host__ __device__ constexpr int cx(int i) {
  constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return v[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return v[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) {
  return i == 0 ? (1.0f / 3.0f) : (i < 7 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr double wgt_d(int i) {
  return i == 0 ? (1.0 / 3.0) : (i < 7 ? (1.0 / 18.0) : (1.0 / 36.0));
}
// Power-of-two scale of the half-precision deviation store, ~1/w_i.
__host__ __device__ constexpr float dev_scale(int i) { return i == 0 ? 4.0f : (i < 7 ? 16.0f : 32.0f); }

enum Geometry : int { GEOM_PERIODIC = 0, GEOM_YWALLS = 1, GEOM_TUBE = 2 };
enum Storage : int { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

// Tiles used to mark where markers touch the lattice: 32 (x) x 4 x 4 cells.
constexpr int TILE_X_SHIFT = 5, TILE_Y_SHIFT = 2, TILE_Z_SHIFT = 2;

struct LatticeDev {
  int nx, ny, nz;
  int N;                 // nx*ny*nz (< 2^31)
  int geometry;
  float omega;           // 1/tau
  float guo_pre;         // 1 - 1/(2 tau)
  float wall_u0, wall_u1;
  float yc, zc, R2;      // tube axis and squared radius
  float g0x, g0y, g0z;   // uniform body force density
  int ntx, nty, ntz;     // tile grid
  void* pop;             // [19][N] in the storage type
  float4* uw;            // moments of the last collision: (ux, uy, uz, rho - 1) [N]
  // Force density and touched-tile flags: the step's spreading adds into g
  // (zero at that point) and marks flags, the collision reads g where flags
  // is set, and the interpolation, which sweeps the same boxes of cells
  // afterwards, writes g back to zero there (in its latency-bound box load,
  // not in the bandwidth-bound collision). flags is cleared at the start of
  // each step.
  float4* g;             // spread force density (gx, gy, gz, 0) [N]
  uint8_t* flags;        // [ntx*nty*ntz]: tile touched by a marker stencil this step
  int* status;           // device status word (0 = OK)
};

// One lattice row (fixed y, z; all x) that holds fluid. Solidity depends on
// (y, z) only in every geometry, so a row is all fluid or all solid and the
// collide kernel runs over the fluid rows alone.
struct RowInfo {
  int base;              // idx of (0, y, z)
  int smask;             // bit (dy+1)*3 + (dz+1): the row at (y+dy, z+dz) is solid
  int oyp, oym, ozp, ozm;// wrapped element offsets to the y+-1, z+-1 rows
  int y;
  int trow;              // tile-row offset ntx * ((y >> 2) + nty * (z >> 2))
};

// A contiguous run of markers handled by one thread block in the transfer
// kernels (a body, or part of one, or a run of passive tracers).
struct MarkerGroup {
  int first, count;
  int flags;  // GROUP_FIXED: positions set by a rigid body, not advected
};
constexpr int GROUP_FIXED = 1;

// Solid test of a node with wrapped x and (for walls/tube) raw y, z.
__device__ __forceinline__ bool solid_yz(const LatticeDev& L, int y, int z) {
  if (L.geometry == GEOM_YWALLS) return (unsigned)y >= (unsigned)L.ny;
  if (L.geometry == GEOM_TUBE) {
    if ((unsigned)y >= (unsigned)L.ny || (unsigned)z >= (unsigned)L.nz) return true;
    float dy = (float)y - L.yc, dz = (float)z - L.zc;
    return dy * dy + dz * dz > L.R2;
  }
  return false;
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v = v % n;
  return v < 0 ? v + n : v;
}

// ---- population storage ---------------------------------------------------
template <int S> struct Store;
template <> struct Store<STORE_F32> {
  using T = float;
  template <int I> __device__ static __forceinline__ float ld(const T* p) { return *p; }
  template <int I> __device__ static __forceinline__ void st(T* p, float v) { *p = v; }
};
template <> struct Store<STORE_F16> {
  using T = __half;
  template <int I> __device__ static __forceinline__ float ld(const T* p) {
    return __half2float(*p) * (1.0f / dev_scale(I));
  }
  template <int I> __device__ static __forceinline__ void st(T* p, float v) {
    *p = __float2half_rn(v * dev_scale(I));
  }
};
template <> struct Store<STORE_BF16> {
  using T = __nv_bfloat16;
  template <int I> __device__ static __forceinline__ float ld(const T* p) {
    return __bfloat162float(*p) * (1.0f / dev_scale(I));
  }
  template <int I> __device__ static __forceinline__ void st(T* p, float v) {
    *p = __float2bfloat16_rn(v * dev_scale(I));
  }
};

// ---- markers and bodies ---------------------------------------------------
struct BodyDev {
  int kind;              // 0 membrane, 1 rigid
  int first, count;
  float kBT_p, k_b, k_l, k_g, k_v;
  double kappa, mass, inertia[3];
  double center[3], quat[4], vel[3], omega[3];
  float qmax;  // membranes: largest force contribution component of the last step (0: none yet)
  float l0;    // filaments: rest bond length
};

struct MeshDev {
  int nv, nt, ne;
  // Template topology packed in one buffer of 16-byte-aligned sections:
  // edges ushort4 (a, b, c, d): edge a->b, wing c in the triangle with a->b,
  // d in the other; edge_tris ushort2 (t1, t2): those two triangles;
  // edge_rest float4 (l0, cos theta0, sin theta0, -); tris ushort4 (v0, v1, v2, -); area0 float;
  // per-vertex CSR lists ve_start/ve of (edge << 2 | role a,b,c,d) and
  // vt_start/vt of (triangle << 2 | slot), all unsigned short.
  const unsigned char* packed;
  int packed_bytes;  // multiple of 16
  int off_edges, off_edge_tris, off_edge_rest, off_tris, off_area0, off_ve_start, off_ve, off_vt_start, off_vt;
  int work_floats;   // per-body shared work area: 9 nv + 4 nt words
  float A0, V0;
  float qcap;        // fixed-point force scatter: largest |contribution| in units, such
                     // that a vertex's sum of all its contributions fits in int32
};

struct MarkersDev {
  int M;
  double* X;          // [3][M] positions (FP64, unwrapped)
  float4* U;          // (Ux, Uy, Uz, 0) [M]
  float4* F;          // (Fx, Fy, Fz, 0) [M]
  const double* ref;  // rigid body-frame offsets [3][M]
  // Stencil cache of the current positions: cell[a][k] = floor(X_a,k) and
  // frac[a][k] = X_a,k - floor(X_a,k) rounded once to FP32. Written when the
  // positions change (set_markers, advection) so that the force, spreading
  // and interpolation kernels need no FP64 arithmetic.
  int* cell;          // [3][M]
  float* frac;        // [3][M]
};

// Stencil cache of one marker coordinate: floor and fractional part.
__device__ __forceinline__ void cache_coord(const MarkersDev& m, size_t off, double X) {
  const double f = floor(X);
  m.cell[off] = (int)f;
  m.frac[off] = (float)(X - f);
}

}  // namespace ibm

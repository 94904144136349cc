// Marker forces of the immersed bodies, one thread block per body.
//
// Membranes (Sec. 2.2 of arXiv:1704.04551): F = -dU/dX of Eq.
// membrane-potential, with
//   U_stretch = sum_j [ (kBT l_m / 4p)(3x^2 - 2x^3)/(1 - x) + k_p / l_j ]   (Eq. inPlanePotential)
//               x = l/l_m, l_m = 2 l0 per edge, k_p = 1.25 (kBT/p) l0^2 so that
//               the bond force vanishes at x = 1/2;
//   U_bend    = sum_edges k_b (1 - cos(theta - theta0))                     (Eq. bendingEnergy)
//               theta = signed angle between the outward normals of the two
//               triangles sharing the edge (positive where convex);
//   U_area    = k_g (A - A0)^2 / (2 A0) + sum_t k_l (A_t - A_t0)^2/(2 A_t0) (Eq. areaEnergy)
//   U_volume  = k_v (V - V0)^2 / (2 V0)                                    (Eq. volumeEnergy)
// Positions are FP64; every geometric quantity is built from FP64
// differences rounded once to FP32, all force arithmetic is FP32; the body's
// total area and volume are reduced in FP64. The volume gradient at a vertex
// uses the closed-surface form dV/dx_v = (1/6) sum_{t at v} N_t (N_t the
// triangle's doubled-area normal), which equals (1/6) sum x_{v+1} x x_{v+2}
// for a closed mesh but needs no absolute coordinates.
//
// Rigid bodies (Sec. 2.3, penalty reading of the rigid coupling): each marker
// is tethered to its body-fixed point X^ref = C + R(q) r_k; the fluid receives
// F_k = -kappa (X_k - X^ref); the body receives the reaction, whose force and
// torque drive one explicit Newton-Euler step in FP64:
//   V += F/m; C += V;  w_b += I^-1 (T_b - w_b x I w_b);  q += (0, w)q/2, |q| = 1.
#include "common.cuh"
#include "internal.h"

namespace ibm {

namespace {

constexpr int FORCE_THREADS = 256;

__device__ __forceinline__ float3 f3(double a, double b, double c) {
  return make_float3((float)a, (float)b, (float)c);
}
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// block-wide FP64 sum of n values per thread (result valid in every thread)
template <int K>
__device__ void block_sum(double (&v)[K], double* sh /* [K][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + warp] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[k * 32 + w];
    v[k] = s;
  }
  __syncthreads();
}

__device__ void rigid_body(const MarkersDev& m, BodyDev* B, double* sh) {
  const size_t M = (size_t)m.M;
  double R[3][3];
  {
    const double w = B->quat[0], x = B->quat[1], y = B->quat[2], z = B->quat[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
  }
  const double C0 = B->center[0], C1 = B->center[1], C2 = B->center[2];
  const double kappa = B->kappa;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = B->first + threadIdx.x; k < B->first + B->count; k += blockDim.x) {
    const double r0 = m.ref[k], r1 = m.ref[M + k], r2 = m.ref[2 * M + k];
    const double w0 = R[0][0] * r0 + R[0][1] * r1 + R[0][2] * r2;
    const double w1 = R[1][0] * r0 + R[1][1] * r1 + R[1][2] * r2;
    const double w2 = R[2][0] * r0 + R[2][1] * r1 + R[2][2] * r2;
    const double d0 = m.X[k] - (C0 + w0), d1 = m.X[M + k] - (C1 + w1), d2 = m.X[2 * M + k] - (C2 + w2);
    m.F[k] = make_float4((float)(-kappa * d0), (float)(-kappa * d1), (float)(-kappa * d2), 0.f);
    const double f0 = kappa * d0, f1 = kappa * d1, f2 = kappa * d2;
    acc[0] += f0; acc[1] += f1; acc[2] += f2;
    acc[3] += w1 * f2 - w2 * f1;
    acc[4] += w2 * f0 - w0 * f2;
    acc[5] += w0 * f1 - w1 * f0;
  }
  block_sum<6>(acc, sh);
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      B->vel[a] += acc[a] / B->mass;
      B->center[a] += B->vel[a];
    }
    double wb[3], tb[3], Iw[3];
    for (int a = 0; a < 3; ++a) {
      wb[a] = R[0][a] * B->omega[0] + R[1][a] * B->omega[1] + R[2][a] * B->omega[2];
      tb[a] = R[0][a] * acc[3] + R[1][a] * acc[4] + R[2][a] * acc[5];
    }
    for (int a = 0; a < 3; ++a) Iw[a] = B->inertia[a] * wb[a];
    const double g0 = wb[1] * Iw[2] - wb[2] * Iw[1];
    const double g1 = wb[2] * Iw[0] - wb[0] * Iw[2];
    const double g2 = wb[0] * Iw[1] - wb[1] * Iw[0];
    wb[0] += (tb[0] - g0) / B->inertia[0];
    wb[1] += (tb[1] - g1) / B->inertia[1];
    wb[2] += (tb[2] - g2) / B->inertia[2];
    for (int a = 0; a < 3; ++a) B->omega[a] = R[a][0] * wb[0] + R[a][1] * wb[1] + R[a][2] * wb[2];
    const double w = B->quat[0], x = B->quat[1], y = B->quat[2], z = B->quat[3];
    const double ox = B->omega[0], oy = B->omega[1], oz = B->omega[2];
    double q0 = w + 0.5 * (-ox * x - oy * y - oz * z);
    double q1 = x + 0.5 * (ox * w + oy * z - oz * y);
    double q2 = y + 0.5 * (-ox * z + oy * w + oz * x);
    double q3 = z + 0.5 * (ox * y - oy * x + oz * w);
    const double n = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    B->quat[0] = q0 / n; B->quat[1] = q1 / n; B->quat[2] = q2 / n; B->quat[3] = q3 / n;
  }
}

__device__ void membrane_body(const MarkersDev& m, const BodyDev& B, const MeshDev& mesh, double* sh,
                              unsigned char* dyn) {
  const size_t M = (size_t)m.M;
  const int nv = mesh.nv;
  double* sX = reinterpret_cast<double*>(dyn);         // [3][nv]
  float* sF = reinterpret_cast<float*>(sX + 3 * nv);   // [3][nv]
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int k = B.first + v;
    sX[v] = m.X[k]; sX[nv + v] = m.X[M + k]; sX[2 * nv + v] = m.X[2 * M + k];
    sF[v] = 0.f; sF[nv + v] = 0.f; sF[2 * nv + v] = 0.f;
  }
  __syncthreads();
  // difference of two vertex positions, FP64 then rounded to FP32
  auto dv = [&](int a, int b) { return f3(sX[a] - sX[b], sX[nv + a] - sX[nv + b], sX[2 * nv + a] - sX[2 * nv + b]); };
  auto addF = [&](int v, float3 f) {
    atomicAdd(sF + v, f.x); atomicAdd(sF + nv + v, f.y); atomicAdd(sF + 2 * nv + v, f.z);
  };

  // total area and volume (FP64 reduction), volume relative to vertex 0
  double av[2] = {0.0, 0.0};
  for (int t = threadIdx.x; t < mesh.nt; t += blockDim.x) {
    const int4 T = mesh.tris[t];
    const float3 e1 = dv(T.y, T.x), e2 = dv(T.z, T.x);
    const float3 N = cross(e1, e2);
    av[0] += 0.5 * (double)sqrtf(dot(N, N));
    const double p0x = sX[T.x] - sX[0], p0y = sX[nv + T.x] - sX[nv], p0z = sX[2 * nv + T.x] - sX[2 * nv];
    // p0 . (p1 x p2) = p0 . ((p1 - p0) x (p2 - p0)) for the triangle's own frame
    av[1] += (p0x * (double)N.x + p0y * (double)N.y + p0z * (double)N.z) / 6.0;
  }
  block_sum<2>(av, sh);
  const float cg = B.k_g * (float)((av[0] - (double)mesh.A0) / (double)mesh.A0);
  const float cv = B.k_v * (float)((av[1] - (double)mesh.V0) / (double)mesh.V0);

  // area (local + global) and volume forces, per triangle
  for (int t = threadIdx.x; t < mesh.nt; t += blockDim.x) {
    const int4 T = mesh.tris[t];
    const int vv[3] = {T.x, T.y, T.z};
    const float3 e1 = dv(T.y, T.x), e2 = dv(T.z, T.x);
    const float3 N = cross(e1, e2);
    const float nN = sqrtf(dot(N, N));
    const float At = 0.5f * nN;
    const float At0 = mesh.tri_area0[t];
    const float coef = B.k_l * (At - At0) / At0 + cg;
    const float3 nh = (1.0f / nN) * N;
    const float3 fV = (-cv / 6.0f) * N;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const float3 opp = dv(vv[(s + 2) % 3], vv[(s + 1) % 3]);
      const float3 gA = cross(nh, opp);
      addF(vv[s], (-0.5f * coef) * gA + fV);
    }
  }
  // stretching and bending, per edge
  for (int e = threadIdx.x; e < mesh.ne; e += blockDim.x) {
    const int4 E = mesh.edges[e];
    const float2 rest = mesh.edge_rest[e];
    const float3 ev = dv(E.y, E.x);  // b - a
    const float L2 = dot(ev, ev), l = sqrtf(L2);
    const float l0 = rest.x, x = l / (2.0f * l0);
    const float kp = 1.25f * B.kBT_p * l0 * l0;
    const float dUdl = B.kBT_p * (0.25f / ((1.0f - x) * (1.0f - x)) - 0.25f + x) - kp / L2;
    const float3 fs = (dUdl / l) * ev;
    addF(E.x, fs);
    addF(E.y, -1.0f * fs);
    if (B.k_b != 0.f) {
      const float3 ca = dv(E.z, E.x), da = dv(E.w, E.x), db = dv(E.w, E.y);
      const float3 n1 = cross(ev, ca);
      const float3 n2 = cross(-1.0f * ev, db);
      const float3 mm = cross(n1, n2);
      const float theta = atan2f(dot(mm, ev) / l, dot(n1, n2));
      const float s = B.k_b * sinf(theta - rest.y);
      const float n1s = dot(n1, n1), n2s = dot(n2, n2);
      const float t1 = dot(ca, ev) / L2, t2 = dot(da, ev) / L2;
      const float3 gc = (-l / n1s) * n1, gd = (-l / n2s) * n2;
      const float3 ga = (-(1.0f - t1)) * gc + (-(1.0f - t2)) * gd;
      const float3 gb = (-t1) * gc + (-t2) * gd;
      addF(E.x, -s * ga);
      addF(E.y, -s * gb);
      addF(E.z, -s * gc);
      addF(E.w, -s * gd);
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x)
    m.F[B.first + v] = make_float4(sF[v], sF[nv + v], sF[2 * nv + v], 0.f);
}

}  // namespace

__global__ void __launch_bounds__(FORCE_THREADS) k_forces(MarkersDev m, BodyDev* bodies, MeshDev mesh) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double sh[6 * 32];
  BodyDev* B = bodies + blockIdx.x;
  if (B->kind == 1) rigid_body(m, B, sh);
  else membrane_body(m, *B, mesh, sh, dyn);
}

size_t forces_smem_bytes(int nv) { return (size_t)nv * (3 * sizeof(double) + 3 * sizeof(float)); }

cudaError_t forces_configure(size_t smem_bytes) {
  return cudaFuncSetAttribute(k_forces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

void launch_forces(const MarkersDev& m, BodyDev* bodies, int n_bodies, const MeshDev& mesh, cudaStream_t st) {
  if (n_bodies == 0) return;
  k_forces<<<n_bodies, FORCE_THREADS, forces_smem_bytes(mesh.nv), st>>>(m, bodies, mesh);
}

}  // namespace ibm

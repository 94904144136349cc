// Marker forces of the immersed bodies.
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
// Positions are FP64. Each vertex is loaded once as its offset from the
// body's first vertex, split into an FP32 pair (hi, lo) with hi + lo equal to
// the FP64 offset to ~2^-48 relative; the difference of two vertices is
// (hi_a - hi_b) + (lo_a - lo_b), accurate to FP32 rounding of the difference
// itself, with no FP64 arithmetic (slow on this GPU). All force arithmetic is
// FP32; the body's total area and volume are reduced in FP64. The volume
// gradient at a vertex uses the closed-surface form
// dV/dx_v = (1/6) sum_{t at v} N_t (N_t the triangle's doubled-area normal),
// which equals (1/6) sum x_{v+1} x x_{v+2} for a closed mesh but needs no
// absolute coordinates.
//
// All membranes share one template mesh, so its topology (16-bit packed) is
// staged once in the shared memory of a persistent thread block that then
// works through the bodies, two at a time (one per 512-thread half, with
// named barriers). Templates too large for that layout use one block per
// body with the topology read from global memory.
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

constexpr int RIGID_THREADS = 256;
constexpr int HALF_THREADS = 512;     // threads per body in the persistent membrane kernel
constexpr int GLOBAL_THREADS = 256;   // threads per body in the fallback membrane kernel

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// barrier over the nthr threads of one body's group
__device__ __forceinline__ void group_sync(int id, int nthr) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
}

// Views of the packed template topology (in shared or global memory).
struct Topo {
  const ushort4* edges;      // (a, b, c, d)
  const ushort2* edge_tris;  // (t1, t2)
  const float2* edge_rest;   // (l0, theta0)
  const ushort4* tris;       // (v0, v1, v2, -)
  const float* area0;
  const unsigned short* ve_start;  // [nv + 1]
  const unsigned short* ve;        // (edge << 2) | role
  const unsigned short* vt_start;  // [nv + 1]
  const unsigned short* vt;        // (triangle << 2) | slot
};

__device__ __forceinline__ Topo topo_at(const unsigned char* base, const MeshDev& mesh) {
  Topo T;
  T.edges = reinterpret_cast<const ushort4*>(base + mesh.off_edges);
  T.edge_tris = reinterpret_cast<const ushort2*>(base + mesh.off_edge_tris);
  T.edge_rest = reinterpret_cast<const float2*>(base + mesh.off_edge_rest);
  T.tris = reinterpret_cast<const ushort4*>(base + mesh.off_tris);
  T.area0 = reinterpret_cast<const float*>(base + mesh.off_area0);
  T.ve_start = reinterpret_cast<const unsigned short*>(base + mesh.off_ve_start);
  T.ve = reinterpret_cast<const unsigned short*>(base + mesh.off_ve);
  T.vt_start = reinterpret_cast<const unsigned short*>(base + mesh.off_vt_start);
  T.vt = reinterpret_cast<const unsigned short*>(base + mesh.off_vt);
  return T;
}

// Membrane forces of one body by a group of nthr threads (thread tid in the
// group, barrier id bar), in three passes over shared memory with no
// atomics (the result does not depend on thread scheduling):
//   A. per triangle: N_t = (x1 - x0) x (x2 - x0), A_t; the body's total
//      area and volume (FP64 group reduction);
//   B. per edge: the stretching coefficient (dU/dl)/l and the bending
//      coefficient k_b sin(theta - theta0), theta from the two triangles'
//      N_t (already the outward normals n1, n2 of the edge's wings);
//   C. per vertex: the sum over the edges and triangles the vertex belongs
//      to, using the stored coefficients and normals.
// work: [6 nv + 4 nt + 2 ne] floats; red: [2 * 32] doubles.
__device__ void membrane_body(const MarkersDev& m, const BodyDev& B, const MeshDev& mesh, const Topo& T,
                              float* work, double* red, int tid, int nthr, int bar) {
  const size_t M = (size_t)m.M;
  const int nv = mesh.nv, nt = mesh.nt, ne = mesh.ne;
  float* sH = work;            // [3][nv] hi parts of the offsets from vertex 0
  float* sL = sH + 3 * nv;     // [3][nv] lo parts
  float* sN = sL + 3 * nv;     // [3][nt] doubled-area normals
  float* sA = sN + 3 * nt;     // [nt] areas
  float* sEs = sA + nt;        // [ne] stretching coefficients
  float* sEb = sEs + ne;       // [ne] bending coefficients
  const double ax0 = m.X[B.first], ay0 = m.X[M + B.first], az0 = m.X[2 * M + B.first];
  for (int v = tid; v < nv; v += nthr) {
    const int k = B.first + v;
    const double o[3] = {m.X[k] - ax0, m.X[M + k] - ay0, m.X[2 * M + k] - az0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float hi = (float)o[a];
      sH[a * nv + v] = hi;
      sL[a * nv + v] = (float)(o[a] - (double)hi);
    }
  }
  group_sync(bar, nthr);
  auto dv = [&](int a, int b) {
    return make_float3((sH[a] - sH[b]) + (sL[a] - sL[b]), (sH[nv + a] - sH[nv + b]) + (sL[nv + a] - sL[nv + b]),
                       (sH[2 * nv + a] - sH[2 * nv + b]) + (sL[2 * nv + a] - sL[2 * nv + b]));
  };
  auto normal = [&](int t) { return make_float3(sN[t], sN[nt + t], sN[2 * nt + t]); };

  // A. triangle normals and areas, total area and volume
  float a_part = 0.f, v_part = 0.f;
  for (int t = tid; t < nt; t += nthr) {
    const ushort4 Tr = T.tris[t];
    const float3 N = cross(dv(Tr.y, Tr.x), dv(Tr.z, Tr.x));
    const float At = 0.5f * sqrtf(dot(N, N));
    sN[t] = N.x; sN[nt + t] = N.y; sN[2 * nt + t] = N.z;
    sA[t] = At;
    a_part += At;
    // p0 . (p1 x p2) = p0 . ((p1 - p0) x (p2 - p0)), p0 the offset of the
    // triangle's first vertex from vertex 0
    const float3 p0 = make_float3(sH[Tr.x] + sL[Tr.x], sH[nv + Tr.x] + sL[nv + Tr.x], sH[2 * nv + Tr.x] + sL[2 * nv + Tr.x]);
    v_part += dot(p0, N) * (1.0f / 6.0f);
  }
  double s0 = a_part, s1 = v_part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((tid & 31) == 0) {
    red[2 * (tid >> 5)] = s0;
    red[2 * (tid >> 5) + 1] = s1;
  }
  group_sync(bar, nthr);  // normals, areas and partial sums are visible
  double A = 0.0, V = 0.0;
  for (int w = 0; w < (nthr >> 5); ++w) {
    A += red[2 * w];
    V += red[2 * w + 1];
  }
  const float cg = B.k_g * (float)((A - (double)mesh.A0) / (double)mesh.A0);
  const float cv = B.k_v * (float)((V - (double)mesh.V0) / (double)mesh.V0);

  // B. per-edge coefficients
  for (int e = tid; e < ne; e += nthr) {
    const ushort4 E = T.edges[e];
    const ushort2 ET = T.edge_tris[e];
    const float2 rest = T.edge_rest[e];
    const float3 ev = dv(E.y, E.x);  // b - a
    const float L2 = dot(ev, ev), l = sqrtf(L2);
    const float l0 = rest.x, x = l / (2.0f * l0);
    const float kp = 1.25f * B.kBT_p * l0 * l0;  // zero bond force at x = 1/2
    const float dUdl = B.kBT_p * (0.25f / ((1.0f - x) * (1.0f - x)) - 0.25f + x) - kp / L2;
    sEs[e] = dUdl / l;
    float sb = 0.f;
    if (B.k_b != 0.f) {
      const float3 n1 = normal(ET.x), n2 = normal(ET.y);
      const float theta = atan2f(dot(cross(n1, n2), ev) / l, dot(n1, n2));
      sb = B.k_b * sinf(theta - rest.y);
    }
    sEb[e] = sb;
  }
  group_sync(bar, nthr);

  // C. per-vertex gather
  for (int v = tid; v < nv; v += nthr) {
    float3 F = make_float3(0.f, 0.f, 0.f);
    for (int q = T.ve_start[v]; q < T.ve_start[v + 1]; ++q) {
      const int code = T.ve[q];
      const int e = code >> 2, role = code & 3;
      const ushort4 E = T.edges[e];
      const float3 ev = dv(E.y, E.x);
      if (role == 0) F = F + sEs[e] * ev;          // stretching: F_a = (dU/dl)/l (b - a)
      else if (role == 1) F = F + (-sEs[e]) * ev;  // F_b = -F_a
      const float s = sEb[e];
      if (s == 0.f) continue;
      // bending: F_v = -s dtheta/dv with dtheta/dc = -L n1/|n1|^2,
      // dtheta/dd = -L n2/|n2|^2, dtheta/da = -(1-t1) g_c - (1-t2) g_d,
      // dtheta/db = -t1 g_c - t2 g_d, t1,2 = (c,d - a).(b - a)/L^2
      const ushort2 ET = T.edge_tris[e];
      const float L2 = dot(ev, ev), l = sqrtf(L2);
      const float3 n1 = normal(ET.x), n2 = normal(ET.y);
      const float3 gc = (-l / dot(n1, n1)) * n1, gd = (-l / dot(n2, n2)) * n2;
      float3 g;
      if (role == 2) {
        g = gc;
      } else if (role == 3) {
        g = gd;
      } else {
        const float t1 = dot(dv(E.z, E.x), ev) / L2, t2 = dot(dv(E.w, E.x), ev) / L2;
        g = (role == 0) ? (-(1.0f - t1)) * gc + (-(1.0f - t2)) * gd : (-t1) * gc + (-t2) * gd;
      }
      F = F + (-s) * g;
    }
    for (int q = T.vt_start[v]; q < T.vt_start[v + 1]; ++q) {
      const int code = T.vt[q];
      const int t = code >> 2, slot = code & 3;
      const ushort4 Tr = T.tris[t];
      const int vv[3] = {Tr.x, Tr.y, Tr.z};
      const float3 N = normal(t);
      // area (local + global): F_v = -coef dA_t/dx_v, dA_t/dx_v = 1/2 n x (x_{v+2} - x_{v+1})
      const float At0 = T.area0[t];
      const float coef = B.k_l * (sA[t] - At0) / At0 + cg;
      const float3 nh = (1.0f / (2.0f * sA[t])) * N;
      const float3 gA = cross(nh, dv(vv[(slot + 2) % 3], vv[(slot + 1) % 3]));
      // volume: F_v = -(k_v (V - V0)/V0) dV/dx_v, dV/dx_v = N_t / 6 summed over the triangles at v
      F = F + (-0.5f * coef) * gA + (-cv / 6.0f) * N;
    }
    m.F[B.first + v] = make_float4(F.x, F.y, F.z, 0.f);
  }
  group_sync(bar, nthr);  // the work area is reused by the next body
}

}  // namespace

// Persistent membrane kernel: 2 x HALF_THREADS threads per block, the
// template topology in shared memory, one body per half at a time.
__global__ void __launch_bounds__(2 * HALF_THREADS, 1)
    k_membranes(MarkersDev m, const BodyDev* __restrict__ bodies, const int* __restrict__ list, int n, MeshDev mesh) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2][2 * 32];
  // stage the packed topology (16-byte words)
  {
    const int4* src = reinterpret_cast<const int4*>(mesh.packed);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < mesh.packed_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const Topo T = topo_at(smem, mesh);
  const int half = threadIdx.x / HALF_THREADS, tid = threadIdx.x % HALF_THREADS;
  float* work = reinterpret_cast<float*>(smem + mesh.packed_bytes) + (size_t)half * mesh.work_floats;
  for (int i = 2 * blockIdx.x + half; i < n; i += 2 * gridDim.x)
    membrane_body(m, bodies[list[i]], mesh, T, work, red[half], tid, HALF_THREADS, 1 + half);
}

// Fallback: one block per membrane, topology read from global memory.
__global__ void __launch_bounds__(GLOBAL_THREADS)
    k_membranes_global(MarkersDev m, const BodyDev* __restrict__ bodies, const int* __restrict__ list, MeshDev mesh) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * 32];
  const Topo T = topo_at(mesh.packed, mesh);
  membrane_body(m, bodies[list[blockIdx.x]], mesh, T, reinterpret_cast<float*>(smem), red, threadIdx.x,
                GLOBAL_THREADS, 1);
}

// One block per rigid body.
__global__ void __launch_bounds__(RIGID_THREADS)
    k_rigid(MarkersDev m, BodyDev* __restrict__ bodies, const int* __restrict__ list) {
  __shared__ double sh[6 * 32];
  BodyDev* B = bodies + list[blockIdx.x];
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
  // block reduction of the body's force and torque
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (lane == 0)
    for (int k = 0; k < 6; ++k) sh[k * 32 + warp] = acc[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 6; ++k) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[k * 32 + w];
    acc[k] = s;
  }
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
  const double q0 = w + 0.5 * (-ox * x - oy * y - oz * z);
  const double q1 = x + 0.5 * (ox * w + oy * z - oz * y);
  const double q2 = y + 0.5 * (-ox * z + oy * w + oz * x);
  const double q3 = z + 0.5 * (ox * y - oy * x + oz * w);
  const double nq = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  B->quat[0] = q0 / nq; B->quat[1] = q1 / nq; B->quat[2] = q2 / nq; B->quat[3] = q3 / nq;
}

size_t membrane_work_floats(int nv, int nt, int ne) { return (size_t)6 * nv + (size_t)4 * nt + (size_t)2 * ne; }

cudaError_t forces_configure(const MeshDev& mesh, size_t max_smem, bool* persistent) {
  const size_t work = sizeof(float) * mesh.work_floats;
  const size_t persistent_smem = (size_t)mesh.packed_bytes + 2 * work;
  *persistent = persistent_smem + 2048 <= max_smem;
  if (*persistent)
    return cudaFuncSetAttribute(k_membranes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persistent_smem);
  if (work + 1024 > max_smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_membranes_global, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work);
}

void launch_forces(const MarkersDev& m, BodyDev* bodies, const int* membranes, int n_membranes, const int* rigids,
                   int n_rigids, const MeshDev& mesh, bool persistent, int n_sm, cudaStream_t st) {
  if (n_rigids > 0) k_rigid<<<n_rigids, RIGID_THREADS, 0, st>>>(m, bodies, rigids);
  if (n_membranes == 0) return;
  const size_t work = sizeof(float) * mesh.work_floats;
  if (persistent) {
    int grid = (n_membranes + 1) / 2;
    if (grid > n_sm) grid = n_sm;
    k_membranes<<<grid, 2 * HALF_THREADS, (size_t)mesh.packed_bytes + 2 * work, st>>>(m, bodies, membranes,
                                                                                       n_membranes, mesh);
  } else {
    k_membranes_global<<<n_membranes, GLOBAL_THREADS, work, st>>>(m, bodies, membranes, mesh);
  }
}

}  // namespace ibm

// Device-side bodies of the marker-force kernels, shared by the
// single-lattice kernels (forces.cu) and the batched serving kernels
// (serve.cu). Marker forces of the immersed bodies.
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
// Positions are FP64; this kernel reads them through the per-marker stencil
// cache (floor(X) as integers, X - floor(X) rounded once to FP32): the
// difference of two vertices is (floor_a - floor_b) + (frac_a - frac_b),
// accurate to FP32 rounding of the difference itself, with no FP64
// arithmetic (slow on this GPU). The integer parts are kept in shared memory
// as floats relative to the body's first vertex (exact, and no conversion
// per difference). All force arithmetic is FP32, with the approximate
// division (2 ulp) where the quotient only scales a force; the body's
// total area and volume are reduced in FP64. The volume gradient at a vertex
// uses the closed-surface form dV/dx_v = (1/6) sum_{t at v} N_t (N_t the
// triangle's doubled-area normal), which equals (1/6) sum x_{v+1} x x_{v+2}
// for a closed mesh but needs no absolute coordinates.
//
// One thread block per membrane. Pass A computes every triangle's normal and
// area and the body's area and volume; pass B adds each edge's stretching
// and bending forces and each triangle's area and volume forces to the
// vertices with shared-memory atomics (fixed point, see membrane_block). All membranes share one template
// mesh; its 16-bit packed topology is read from global memory and stays in
// the L1 cache.
//
// Rigid bodies (Sec. 2.3, penalty reading of the rigid coupling): each marker
// is tethered to its body-fixed point X^ref = C + R(q) r_k; the fluid receives
// F_k = -kappa (X_k - X^ref); the body receives the reaction, whose force and
// torque drive one explicit Newton-Euler step in FP64:
//   V += F/m; C += V;  w_b += I^-1 (T_b - w_b x I w_b);  q += (0, w)q/2, |q| = 1.
#pragma once
#include "common.cuh"

namespace ibm {

namespace forces_detail {

constexpr int RIGID_THREADS = 256;
constexpr int MEMBRANE_THREADS = 256;
constexpr int FILAMENT_THREADS = 64;

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Views of the packed template topology.
struct Topo {
  const ushort4* edges;      // (a, b, c, d)
  const ushort2* edge_tris;  // (t1, t2)
  const float4* edge_rest;   // (l0, cos theta0, sin theta0, -)
  const ushort4* tris;       // (v0, v1, v2, -)
  const float* area0;
};

__device__ __forceinline__ Topo topo_at(const unsigned char* base, const MeshDev& mesh) {
  Topo T;
  T.edges = reinterpret_cast<const ushort4*>(base + mesh.off_edges);
  T.edge_tris = reinterpret_cast<const ushort2*>(base + mesh.off_edge_tris);
  T.edge_rest = reinterpret_cast<const float4*>(base + mesh.off_edge_rest);
  T.tris = reinterpret_cast<const ushort4*>(base + mesh.off_tris);
  T.area0 = reinterpret_cast<const float*>(base + mesh.off_area0);
  return T;
}

}  // namespace forces_detail
using namespace forces_detail;

// Shared-memory views of the membrane force core: vertex positions as
// integer part (floats, relative to any common origin: exact) and fraction,
// force sums, triangle normals and areas.
struct MembraneSmem {
  float* sI;  // [3][nv]
  float* sR;  // [3][nv]
  int* sQ;    // [3][nv] force sums (fixed point, or float bits); on return the forces as floats
  float* sN;  // [3][nt] doubled-area normals
  float* sA;  // [nt] areas
  __device__ static MembraneSmem at(unsigned char* base, int nv, int nt) {
    MembraneSmem S;
    S.sI = reinterpret_cast<float*>(base);
    S.sR = S.sI + 3 * nv;
    S.sQ = reinterpret_cast<int*>(S.sR + 3 * nv);
    S.sN = reinterpret_cast<float*>(S.sQ + 3 * nv);
    S.sA = S.sN + 3 * nt;
    return S;
  }
};

// The per-vertex force sums membrane_core leaves in S.sQ [3][nv]: fixed-point
// integers in units of `unit`, or float bits after the float redo.
struct ForceSums {
  const int* q;
  bool is_float;
  float unit;
  __device__ __forceinline__ float operator()(int i) const {
    return is_float ? __int_as_float(q[i]) : (float)q[i] * unit;
  }
};

__device__ __forceinline__ ForceSums membrane_core(BodyDev* Bp, const MeshDev& mesh, const MembraneSmem& S,
                                                   double* red);

// Membrane forces of one body by the whole thread block. smem: [9 nv + 4 nt]
// words (positions as floor + fraction, force sums, normals, areas);
// red: [2 * 32] doubles.
//
// The force sums are scattered with shared-memory integer atomics in fixed
// point (native and order-independent; float atomics on shared memory are
// several times slower): each contribution is scaled by Sq = qcap / (4 q),
// q the body's largest contribution component of the previous step, so that
// contributions up to four times larger than last step's fit in qcap units
// and no vertex sum can overflow. A block that meets a larger contribution,
// or has no previous step, redoes the scatter with float atomics. The
// quantum 1/Sq is ~3e-8 q, below the FP32 rounding of the sums.
__device__ __forceinline__ void membrane_block(const MarkersDev& m, BodyDev* Bp, const MeshDev& mesh,
                                               unsigned char* smem, double* red) {
  const size_t M = (size_t)m.M;
  const int nv = mesh.nv;
  const MembraneSmem S = MembraneSmem::at(smem, nv, mesh.nt);
  const int first = Bp->first;
  const int c0[3] = {m.cell[first], m.cell[M + first], m.cell[2 * M + first]};
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S.sI[a * nv + v] = (float)(m.cell[a * M + first + v] - c0[a]);
      S.sR[a * nv + v] = m.frac[a * M + first + v];
    }
  }
  __syncthreads();
  const ForceSums F = membrane_core(Bp, mesh, S, red);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) m.F[first + v] = make_float4(F(v), F(nv + v), F(2 * nv + v), 0.f);
}

// Forces of one membrane whose positions are in S.sI / S.sR (the caller has
// synchronised after writing them): S.sQ receives the per-vertex sums
// [3][nv] (read through the returned ForceSums), Bp->qmax the scale for the
// next step; ends synchronised.
__device__ __forceinline__ ForceSums membrane_core(BodyDev* Bp, const MeshDev& mesh, const MembraneSmem& S,
                                                   double* red) {
  const Topo T = topo_at(mesh.packed, mesh);
  const int nv = mesh.nv, nt = mesh.nt, ne = mesh.ne;
  const float kBT_p = Bp->kBT_p, k_b = Bp->k_b, k_l = Bp->k_l, k_g = Bp->k_g, k_v = Bp->k_v;
  const float q_prev = Bp->qmax;
  const float* sI = S.sI;
  const float* sR = S.sR;
  int* sQ = S.sQ;
  float* sN = S.sN;
  float* sA = S.sA;
  __shared__ float s_dev[2];
  __shared__ unsigned s_qmax;
  for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) sQ[i] = 0;
  if (threadIdx.x == 0) s_qmax = 0u;
  // x_a - x_b, exact in the integer part, one FP32 rounding in the fraction
  auto dv = [&](int a, int b) {
    return make_float3((sI[a] - sI[b]) + (sR[a] - sR[b]), (sI[nv + a] - sI[nv + b]) + (sR[nv + a] - sR[nv + b]),
                       (sI[2 * nv + a] - sI[2 * nv + b]) + (sR[2 * nv + a] - sR[2 * nv + b]));
  };
  auto normal = [&](int t) { return make_float3(sN[t], sN[nt + t], sN[2 * nt + t]); };

  // A. triangle normals and areas, total area and volume
  float a_part = 0.f, v_part = 0.f;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const ushort4 Tr = T.tris[t];
    const float3 N = cross(dv(Tr.y, Tr.x), dv(Tr.z, Tr.x));
    const float At = 0.5f * sqrtf(dot(N, N));
    sN[t] = N.x; sN[nt + t] = N.y; sN[2 * nt + t] = N.z;
    sA[t] = At;
    a_part += At;
    // p0 . (p1 x p2) = p0 . ((p1 - p0) x (p2 - p0)), p0 the offset of the
    // triangle's first vertex from vertex 0
    v_part += dot(dv(Tr.x, 0), N) * (1.0f / 6.0f);
  }
  double s0 = a_part, s1 = v_part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = s0;
    red[2 * (threadIdx.x >> 5) + 1] = s1;
  }
  __syncthreads();  // normals, areas and partial sums are visible
  if (threadIdx.x == 0) {
    // A - A0 and V - V0 in FP64 (small differences of large sums)
    double A = 0.0, V = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      A += red[2 * w];
      V += red[2 * w + 1];
    }
    s_dev[0] = (float)(A - (double)mesh.A0) / mesh.A0;
    s_dev[1] = (float)(V - (double)mesh.V0) / mesh.V0;
  }
  __syncthreads();
  const float cg = k_g * s_dev[0];
  const float cv = k_v * s_dev[1];

  // B. stretching and bending per edge, area and volume per triangle, each
  // contribution handed to `add`
  float qmax = 0.f;  // largest contribution component seen by this thread
  auto pass_b = [&](auto&& add) {
    // the next edge's topology is loaded while this one is computed
    ushort4 En = make_ushort4(0, 0, 0, 0);
    float4 rn = make_float4(0.f, 0.f, 0.f, 0.f);
    ushort2 ETn = make_ushort2(0, 0);
    if ((int)threadIdx.x < ne) {
      En = T.edges[threadIdx.x];
      rn = T.edge_rest[threadIdx.x];
      ETn = T.edge_tris[threadIdx.x];
    }
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const ushort4 E = En;
      const float4 rest = rn;
      const ushort2 ET = ETn;
      if (e + (int)blockDim.x < ne) {
        En = T.edges[e + blockDim.x];
        rn = T.edge_rest[e + blockDim.x];
        ETn = T.edge_tris[e + blockDim.x];
      }
      const float3 ev = dv(E.y, E.x);  // b - a
      const float L2 = dot(ev, ev), l = sqrtf(L2);
      const float rL2 = __fdividef(1.0f, L2), rl = l * rL2;
      const float l0 = rest.x, x = __fdividef(l, 2.0f * l0);
      const float kp = 1.25f * kBT_p * l0 * l0;  // zero bond force at x = 1/2
      const float dUdl = kBT_p * (__fdividef(0.25f, (1.0f - x) * (1.0f - x)) - 0.25f + x) - kp * rL2;
      const float3 fs = (dUdl * rl) * ev;  // F_a = (dU/dl)/l (b - a), F_b = -F_a
      if (k_b == 0.f) {
        add(E.x, fs);
        add(E.y, (-1.0f) * fs);
        continue;
      }
      // bending: F_v = -s dtheta/dv with dtheta/dc = -L n1/|n1|^2,
      // dtheta/dd = -L n2/|n2|^2, dtheta/da = -(1-t1) g_c - (1-t2) g_d,
      // dtheta/db = -t1 g_c - t2 g_d, t1,2 = (c,d - a).(b - a)/L^2
      const float3 n1 = normal(ET.x), n2 = normal(ET.y);
      // sin(theta - theta0) = sin(theta) cos(theta0) - cos(theta) sin(theta0), with
      // cos(theta), sin(theta) from the normals (no inverse trigonometry)
      const float inv = rsqrtf(dot(n1, n1) * dot(n2, n2));
      const float cth = dot(n1, n2) * inv, sth = dot(cross(n1, n2), ev) * rl * inv;
      const float sb = k_b * (sth * rest.y - cth * rest.z);
      const float3 gc = __fdividef(-l, dot(n1, n1)) * n1, gd = __fdividef(-l, dot(n2, n2)) * n2;
      const float t1 = dot(dv(E.z, E.x), ev) * rL2, t2 = dot(dv(E.w, E.x), ev) * rL2;
      add(E.x, fs + (sb * (1.0f - t1)) * gc + (sb * (1.0f - t2)) * gd);
      add(E.y, (-1.0f) * fs + (sb * t1) * gc + (sb * t2) * gd);
      add(E.z, (-sb) * gc);
      add(E.w, (-sb) * gd);
    }
    ushort4 Trn = make_ushort4(0, 0, 0, 0);
    float A0n = 1.f;
    if ((int)threadIdx.x < nt) {
      Trn = T.tris[threadIdx.x];
      A0n = T.area0[threadIdx.x];
    }
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      const ushort4 Tr = Trn;
      const float At0 = A0n;
      if (t + (int)blockDim.x < nt) {
        Trn = T.tris[t + blockDim.x];
        A0n = T.area0[t + blockDim.x];
      }
      const int vv[3] = {Tr.x, Tr.y, Tr.z};
      const float3 N = normal(t);
      const float At = sA[t];
      const float coef = k_l * __fdividef(At - At0, At0) + cg;
      const float3 nh = __fdividef(0.5f, At) * N;
      const float3 fV = (-cv / 6.0f) * N;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        // F_v = -coef dA_t/dx_v - (k_v (V - V0)/V0) N_t / 6, dA_t/dx_v = 1/2 n x (x_{v+2} - x_{v+1})
        const float3 gA = cross(nh, dv(vv[(q + 2) % 3], vv[(q + 1) % 3]));
        add(vv[q], (-0.5f * coef) * gA + fV);
      }
    }
  };
  const float Sq = q_prev > 0.f ? mesh.qcap / (4.0f * q_prev) : 0.f;
  bool over = !(q_prev > 0.f);
  if (!over) {
    pass_b([&](int v, float3 f) {
      const float c = fmaxf(fabsf(f.x), fmaxf(fabsf(f.y), fabsf(f.z)));
      qmax = fmaxf(qmax, c);
      // a contribution above the headroom (or not finite) sends the block to
      // the float redo, which discards these sums: no branch here
      over |= !(c * Sq <= mesh.qcap);
      atomicAdd(sQ + v, __float2int_rn(f.x * Sq));
      atomicAdd(sQ + nv + v, __float2int_rn(f.y * Sq));
      atomicAdd(sQ + 2 * nv + v, __float2int_rn(f.z * Sq));
    });
  }
  const bool fallback = __syncthreads_or(over) != 0;
  if (fallback) {
    float* sF = reinterpret_cast<float*>(sQ);
    for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) sF[i] = 0.f;
    __syncthreads();
    pass_b([&](int v, float3 f) {
      qmax = fmaxf(qmax, fmaxf(fabsf(f.x), fmaxf(fabsf(f.y), fabsf(f.z))));
      atomicAdd(sF + v, f.x);
      atomicAdd(sF + nv + v, f.y);
      atomicAdd(sF + 2 * nv + v, f.z);
    });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&s_qmax, __float_as_uint(qmax));  // non-negative floats order as their bits
  __syncthreads();  // the sums and s_qmax are complete
  if (threadIdx.x == 0) {
    const float q = __uint_as_float(s_qmax);
    Bp->qmax = isfinite(q) ? q : 0.f;
  }
  ForceSums F;
  F.q = sQ;
  F.is_float = fallback;
  F.unit = fallback ? 0.f : 1.0f / Sq;
  return F;
}

// Filament forces of one bead chain (polymer particles, Sec. 2.2) by the
// whole thread block, one thread per bead: every bead gathers the terms
// that involve it (its two bonds, the angle at itself and at each
// neighbour), so no bead is written twice and no atomics are needed.
//   bond (Eq. inPlanePotential): l_m = 2 l0, k_p = 1.25 (kBT/p) l0^2;
//   angle (Eq. bendingEnergyWorm): U = k_b (theta - pi)^2, theta the angle
//   between the two bonds at an interior bead; with cos(theta) = u.v/(|u||v|),
//   u, v the bonds to the previous and next bead,
//   dU/dcos = 2 k_b phi / sin(phi), phi = pi - theta (limit 2 k_b when straight),
//   F_prev = -dU/dcos dcos/du, F_next = -dU/dcos dcos/dv, F_mid = -(F_prev + F_next).
namespace forces_detail {

// X_a - X_b from the stencil cache: exact integer part, one FP32 rounding
__device__ __forceinline__ float3 marker_diff(const MarkersDev& m, int a, int b) {
  const size_t M = (size_t)m.M;
  return make_float3((float)(m.cell[a] - m.cell[b]) + (m.frac[a] - m.frac[b]),
                     (float)(m.cell[M + a] - m.cell[M + b]) + (m.frac[M + a] - m.frac[M + b]),
                     (float)(m.cell[2 * M + a] - m.cell[2 * M + b]) + (m.frac[2 * M + a] - m.frac[2 * M + b]));
}

// d cos(theta) / du and / dv for bonds u, v of one angle, and dU/dcos
struct AngleGrad {
  float3 du, dv;
  float g;
};
__device__ __forceinline__ AngleGrad angle_grad(float3 u, float3 v, float k_b) {
  const float lu = sqrtf(dot(u, u)), lv = sqrtf(dot(v, v));
  const float3 w = cross(u, v);
  const float sw = sqrtf(dot(w, w)), c = dot(u, v);
  const float inv = 1.0f / (lu * lv), cs = c * inv, sn = sw * inv;
  const float phi = atan2f(sw, -c);  // pi - theta
  const float ratio = sn > 1e-6f ? phi / sn : 1.0f + phi * phi * (1.0f / 6.0f);
  AngleGrad G;
  G.g = 2.0f * k_b * ratio;
  G.du = inv * v + (-cs / (lu * lu)) * u;
  G.dv = inv * u + (-cs / (lv * lv)) * v;
  return G;
}

}  // namespace forces_detail

__device__ __forceinline__ void filament_block(const MarkersDev& m, const BodyDev& B) {
  const int n = B.count, f = B.first;
  const float l0 = B.l0, kBT_p = B.kBT_p, k_b = B.k_b;
  const float kp = 1.25f * kBT_p * l0 * l0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float3 F = make_float3(0.f, 0.f, 0.f);
    // bonds j-1 -> j and j -> j+1: F_j += dU/dl (X_other - X_j)/l
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
      const int o = j + side;
      if (o < 0 || o >= n) continue;
      const float3 e = marker_diff(m, f + o, f + j);
      const float L2 = dot(e, e), l = sqrtf(L2), x = l / (2.0f * l0);
      const float dUdl = kBT_p * (0.25f / ((1.0f - x) * (1.0f - x)) - 0.25f + x) - kp / L2;
      F = F + (dUdl / l) * e;
    }
    if (k_b != 0.f) {
      // angle at j itself
      if (j >= 1 && j + 1 < n) {
        const AngleGrad G = angle_grad(marker_diff(m, f + j - 1, f + j), marker_diff(m, f + j + 1, f + j), k_b);
        F = F + G.g * (G.du + G.dv);
      }
      // angle at j - 1: j is its next bead
      if (j >= 2) {
        const AngleGrad G = angle_grad(marker_diff(m, f + j - 2, f + j - 1), marker_diff(m, f + j, f + j - 1), k_b);
        F = F + (-G.g) * G.dv;
      }
      // angle at j + 1: j is its previous bead
      if (j + 2 < n) {
        const AngleGrad G = angle_grad(marker_diff(m, f + j, f + j + 1), marker_diff(m, f + j + 2, f + j + 1), k_b);
        F = F + (-G.g) * G.du;
      }
    }
    m.F[f + j] = make_float4(F.x, F.y, F.z, 0.f);
  }
}

__device__ __forceinline__ void rigid_update(BodyDev* B, const double R[3][3], const double* sh);

// Tether forces and Newton-Euler update of one rigid body by the whole
// thread block. sh: [6 * 32] doubles.
__device__ __forceinline__ void rigid_block(const MarkersDev& m, BodyDev* B, double* sh) {
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
  const bool direct = B->kind == 3;
  const double V0 = B->vel[0], V1 = B->vel[1], V2 = B->vel[2];
  const double O0 = B->omega[0], O1 = B->omega[1], O2 = B->omega[2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = B->first + threadIdx.x; k < B->first + B->count; k += blockDim.x) {
    const double r0 = m.ref[k], r1 = m.ref[M + k], r2 = m.ref[2 * M + k];
    const double w0 = R[0][0] * r0 + R[0][1] * r1 + R[0][2] * r2;
    const double w1 = R[1][0] * r0 + R[1][1] * r1 + R[1][2] * r2;
    const double w2 = R[2][0] * r0 + R[2][1] * r1 + R[2][2] * r2;
    double f0, f1, f2;  // force on the solid
    if (direct) {
      // Eq. FSIRigid: kappa (u(X) - (V + omega x r)), u the last interpolated velocity
      const float4 u = m.U[k];
      f0 = kappa * ((double)u.x - (V0 + O1 * w2 - O2 * w1));
      f1 = kappa * ((double)u.y - (V1 + O2 * w0 - O0 * w2));
      f2 = kappa * ((double)u.z - (V2 + O0 * w1 - O1 * w0));
    } else {
      f0 = kappa * (m.X[k] - (C0 + w0));
      f1 = kappa * (m.X[M + k] - (C1 + w1));
      f2 = kappa * (m.X[2 * M + k] - (C2 + w2));
    }
    m.F[k] = make_float4((float)(-f0), (float)(-f1), (float)(-f2), 0.f);
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
  if (threadIdx.x == 0) {
    rigid_update(B, R, sh);
    if (direct)  // hand the new pose to the block through shared memory
      for (int a = 0; a < 4; ++a) sh[a] = B->quat[a];
    if (direct)
      for (int a = 0; a < 3; ++a) sh[4 + a] = B->center[a];
  }
  if (!direct) return;
  __syncthreads();
  // direct forcing: the markers follow the body to its new pose
  double Q[3][3];
  {
    const double w = sh[0], x = sh[1], y = sh[2], z = sh[3];
    Q[0][0] = 1 - 2 * (y * y + z * z); Q[0][1] = 2 * (x * y - w * z);     Q[0][2] = 2 * (x * z + w * y);
    Q[1][0] = 2 * (x * y + w * z);     Q[1][1] = 1 - 2 * (x * x + z * z); Q[1][2] = 2 * (y * z - w * x);
    Q[2][0] = 2 * (x * z - w * y);     Q[2][1] = 2 * (y * z + w * x);     Q[2][2] = 1 - 2 * (x * x + y * y);
  }
  const double Cn[3] = {sh[4], sh[5], sh[6]};
  for (int k = B->first + threadIdx.x; k < B->first + B->count; k += blockDim.x) {
    const double r0 = m.ref[k], r1 = m.ref[M + k], r2 = m.ref[2 * M + k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double X = Cn[a] + Q[a][0] * r0 + Q[a][1] * r1 + Q[a][2] * r2;
      m.X[a * M + k] = X;
      cache_coord(m, a * M + k, X);
    }
  }
}

// One explicit Newton-Euler step of a rigid body from the per-warp partial
// sums of its force and torque in sh (thread 0 of the block).
__device__ __forceinline__ void rigid_update(BodyDev* B, const double R[3][3], const double* sh) {
  double acc[6];
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

}  // namespace ibm

// Fused coupling kernel for suspensions of membranes: one thread block per
// membrane body does, between the collision of step n and that of step n+1,
//   1. the interpolation of step n (Eq. ibmVelocityInterpret) from the box of
//      velocities the collision wrote, and the advection X^{n+1} = X^n + U
//      (FP64), clearing the force density the collision consumed;
//   2. the membrane forces at X^{n+1} (Sec. 2.2, Eqs. membrane-potential ..
//      volumeEnergy), from the new positions kept in shared memory;
//   3. the spreading of those forces for step n+1 (Eq. ibmForceSpread) into
//      the other force-density buffer, and the touched tiles of step n+1.
// The arithmetic of each part is that of the separate kernels (the device
// bodies are shared: transfer_group.cuh, forces_body.cuh); what the fusion
// removes is two kernel boundaries, the reloading of the stencil cache and
// of the marker forces between the parts, and the bounding-box pass of the
// spreading. Two force-density buffers are needed: a block clears the one
// the collision of step n read while other blocks already spread into the
// one the collision of step n+1 reads.
//
// Shared memory (the parts reuse one region): the velocity box, the
// gathered velocities and the gather order (part 1); then the vertex
// positions and forces, the triangle normals and areas (part 2); then the
// fixed-point box and the vertex order (part 3), placed after the positions
// and forces, which part 3 still reads. Part 3 also stores its vertex
// order in global memory beside the box, for part 1 of the next step,
// which gathers at the same positions.
#include "common.cuh"
#include "forces_body.cuh"
#include "internal.h"
#include "transfer_group.cuh"

namespace ibm {

// Threads of a fused block (16 warps; 64 registers, two blocks per SM) and
// vertices a thread advects (templates of up to COUPLE_PER_THREAD *
// COUPLE_THREADS vertices take the fused path).
constexpr int COUPLE_THREADS = 512;
constexpr int COUPLE_PER_THREAD = 2;

// End (bytes, rounded to 16) of the largest of the parts' regions: the
// velocity box; the membrane arrays; the positions, forces, fixed-point box
// and vertex order.
__host__ __device__ constexpr int couple_residues_offset(int nv, int nt) {
  const int box = BOX_CELLS * 16;
  const int forces = 36 * nv + 16 * nt;
  const int spread = 36 * nv + 12 * BOX_CELLS + 2 * nv;
  const int most = box > forces ? (box > spread ? box : spread) : (forces > spread ? forces : spread);
  return (most + 15) / 16 * 16;
}

// Part 1 keeps, after the velocity box, the gathered velocities [nv]
// float4 and the gather order [nv] ushort.
__host__ __device__ constexpr int couple_gather_end(int nv) { return BOX_CELLS * 16 + 18 * nv; }

// The counters of the residue sort lie after every region (they are
// cleared at the start and counted from the end of part 1 on).
__host__ __device__ constexpr int couple_counters_offset(int nv, int nt) {
  const int a = couple_residues_offset(nv, nt), b = (couple_gather_end(nv) + 15) / 16 * 16;
  return a > b ? a : b;
}

// Per-body record the spreading leaves for the next step's gather: the
// residue counters (counts [32], starts [32], largest count) of the
// vertices' first stencil nodes in the box it wrote, then the vertex order.
constexpr int ORDER_META_INTS = 68;
__host__ __device__ constexpr int couple_order_stride(int nv) { return (ORDER_META_INTS * 4 + 2 * nv + 15) / 16 * 16; }

namespace {

// Stencil of vertex v from the positions in shared memory (integer parts
// relative to o, fractions).
__device__ __forceinline__ void smem_cell(const MembraneSmem& S, int nv, int v, int3 o, int c[3], float f[3]) {
  c[0] = o.x + (int)S.sI[v];
  c[1] = o.y + (int)S.sI[nv + v];
  c[2] = o.z + (int)S.sI[2 * nv + v];
  f[0] = S.sR[v];
  f[1] = S.sR[nv + v];
  f[2] = S.sR[2 * nv + v];
}

template <int GEOM>
__device__ __forceinline__ void couple_membrane(const LatticeDev& L, float4* g_next, const MarkersDev& m, BodyDev* B,
                                                const MarkerGroup G, int4* box, unsigned char* orec,
                                                const MeshDev& mesh, unsigned char* smem, double* red) {
  __shared__ int s_lo[3], s_hi[3];
  __shared__ unsigned s_fmax;
  const size_t M = (size_t)m.M;
  const int nv = mesh.nv, nt = mesh.nt;  // G.count == nv
  const int4 lo = box[0], dims = box[1];
  const bool in_box = dims.w != 0;
  // lo.w != 0: the previous step's spreading left the residue order of
  // these stencils in this box (orec)
  const bool ordered = in_box && lo.w != 0;
  float4* vbox = reinterpret_cast<float4*>(smem);
  float4* uS = reinterpret_cast<float4*>(smem + BOX_CELLS * 16);         // [nv] gathered velocities
  unsigned short* oS = reinterpret_cast<unsigned short*>(uS + nv);        // [nv] gather order
  const int* ometa = reinterpret_cast<const int*>(orec);
  const unsigned short* oidx = reinterpret_cast<const unsigned short*>(orec + ORDER_META_INTS * 4);
  Residues& R = *reinterpret_cast<Residues*>(smem + couple_counters_offset(nv, nt));
  // origin of the integer parts in shared memory: the first vertex's cell
  // before this step's advection (read before any thread writes the cache)
  const int3 o = make_int3(m.cell[G.first], m.cell[M + G.first], m.cell[2 * M + G.first]);
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;

  // ---- 1. interpolation of step n and advection --------------------------
  // The velocity box loads while the block reads its markers' FP64
  // positions and the gather order. With the order, lane r of a warp gathers
  // for the markers whose first node has box index = r (mod 32), so that
  // the 16-byte loads of a quarter warp fall in distinct banks; without it
  // (the first step after separate kernels) each thread gathers for its own
  // markers. The velocities go to shared memory; after a barrier each thread
  // advects its own markers and writes their positions over the box.
  if (in_box) velocity_box_async<GEOM>(L, lo, dims, vbox);
  // bounds of the new stencils, largest force component, residue counts
  if (threadIdx.x < 3) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
  }
  if (threadIdx.x == 0) s_fmax = 0u;
  if (threadIdx.x < 32) R.cnt[threadIdx.x] = 0;
  double Xo[COUPLE_PER_THREAD][3];
#pragma unroll
  for (int q = 0; q < COUPLE_PER_THREAD; ++q) {
    const int j = threadIdx.x + q * COUPLE_THREADS;
#pragma unroll
    for (int a = 0; a < 3; ++a) Xo[q][a] = j < nv ? m.X[a * M + G.first + j] : 0.0;
  }
  int ocnt = 0, ost = 0, omost = 0;
  if (ordered) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) oS[i] = oidx[i];
    ocnt = ometa[lane];
    ost = ometa[32 + lane];
    omost = ometa[64];
  }
  if (in_box) velocity_box_wait();
  __syncthreads();
  auto gather = [&](int j) {
    Stencil st;
    load_stencil(m, G.first + j, st);
    const int ox = st.bx - lo.x, oy = st.by - lo.y, oz = st.bz - lo.z;
    float3 u;
    if (in_box && ox >= 0 && oy >= 0 && oz >= 0 && ox + 4 <= dims.x && oy + 4 <= dims.y && oz + 4 <= dims.z)
      u = box_gather(vbox, dims, st, ox, oy, oz);
    else  // no box, or the stencil outside it
      u = gather_global<GEOM>(L, st, !in_box);
    uS[j] = make_float4(u.x, u.y, u.z, 0.f);
  };
  if (ordered) {
    for (int w = threadIdx.x >> 5; w < omost; w += nwarps)
      if (w < ocnt) gather(oS[ost + w]);
  } else {
#pragma unroll
    for (int q = 0; q < COUPLE_PER_THREAD; ++q) {
      const int j = threadIdx.x + q * COUPLE_THREADS;
      if (j < nv) gather(j);
    }
  }
  __syncthreads();  // the velocity box is done: the positions go over it
  const MembraneSmem S = MembraneSmem::at(smem, nv, nt);
  const int oa[3] = {o.x, o.y, o.z};
  {
    int l[3] = {INT_MAX, INT_MAX, INT_MAX}, h[3] = {INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
    for (int q = 0; q < COUPLE_PER_THREAD; ++q) {
      const int j = threadIdx.x + q * COUPLE_THREADS;
      if (j >= nv) continue;
      const int k = G.first + j;
      const float4 u = uS[j];
      m.U[k] = u;
      const float ua[3] = {u.x, u.y, u.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double Xn = Xo[q][a] + (double)ua[a];
        m.X[a * M + k] = Xn;
        const double fl = floor(Xn);
        const int c = (int)fl;
        const float f = (float)(Xn - fl);
        m.cell[a * M + k] = c;
        m.frac[a * M + k] = f;
        S.sI[a * nv + j] = (float)(c - oa[a]);
        S.sR[a * nv + j] = f;
        l[a] = min(l[a], c);
        h[a] = max(h[a], c);
      }
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        l[a] = min(l[a], __shfl_xor_sync(0xffffffffu, l[a], w));
        h[a] = max(h[a], __shfl_xor_sync(0xffffffffu, h[a], w));
      }
    if (lane == 0)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        atomicMin(&s_lo[a], l[a]);
        atomicMax(&s_hi[a], h[a]);
      }
  }
  __syncthreads();
  // the stencil box of the new positions (part 3); the vertices are counted
  // by residue now, while the membrane part runs
  const long long ex = (long long)s_hi[0] - s_lo[0] + 4, ey = (long long)s_hi[1] - s_lo[1] + 4,
                  ez = (long long)s_hi[2] - s_lo[2] + 4;
  const bool fits = ex > 0 && ey > 0 && ez > 0 && ex * ey * ez <= BOX_CELLS;
  const int4 dims2 = make_int4(fits ? (int)ex : 0, fits ? (int)ey : 0, fits ? (int)ez : 0, fits ? 1 : 0);
  int l2[COUPLE_PER_THREAD];
#pragma unroll
  for (int q = 0; q < COUPLE_PER_THREAD; ++q) {
    const int v = threadIdx.x + q * COUPLE_THREADS;
    l2[q] = -1;
    if (!fits || v >= nv) continue;
    l2[q] = ((int)S.sI[v] + o.x - s_lo[0]) +
            dims2.x * (((int)S.sI[nv + v] + o.y - s_lo[1]) + dims2.y * ((int)S.sI[2 * nv + v] + o.z - s_lo[2]));
    atomicAdd(&R.cnt[l2[q] & 31], 1);
  }

  // ---- 2. membrane forces at X^{n+1} ---------------------------------------
  const ForceSums sF = membrane_core(B, mesh, S, red);  // ends synchronised
  {
    float fm = 0.f;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const float fx = sF(v), fy = sF(nv + v), fz = sF(2 * nv + v);
      m.F[G.first + v] = make_float4(fx, fy, fz, 0.f);
      fm = fmaxf(fm, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, w));
    if (lane == 0) atomicMax(&s_fmax, __float_as_uint(fm));  // non-negative floats order as their bits
  }
  if (fits) residue_scan(R);  // warp 0; the counts are complete (barriers in the membrane part)
  __syncthreads();

  // ---- 3. spreading of step n+1 into g_next -------------------------------
  const float fmax = __uint_as_float(s_fmax);
  // w = 1: the vertex order of this box is stored in orec below
  const int4 lo2 = make_int4(s_lo[0] - 1, s_lo[1] - 1, s_lo[2] - 1, fits && fmax > 0.f ? 1 : 0);
  if (threadIdx.x == 0) {
    box[0] = lo2;
    box[1] = dims2;
  }
  LatticeDev Ln = L;
  Ln.g = g_next;
  if (!fits) {
    // per-vertex global atomics; touched tiles vertex by vertex (whole warps
    // iterate together: shuffles in mark_tiles)
    for (int j0 = 0; j0 < nv; j0 += blockDim.x) {
      if (j0 + (int)(threadIdx.x & ~31u) >= nv) break;
      const int v = j0 + threadIdx.x;
      const bool active = v < nv;
      const int vv = active ? v : 0;
      int c[3];
      float f[3];
      smem_cell(S, nv, vv, o, c, f);
      Stencil st;
      st.bx = c[0] - 1;
      st.by = c[1] - 1;
      st.bz = c[2] - 1;
      axis_weights(f[0], st.wx);
      axis_weights(f[1], st.wy);
      axis_weights(f[2], st.wz);
      mark_tiles<GEOM>(Ln, st.bx, st.by, st.bz, active);
      if (active && fmax > 0.f)
        scatter_global<GEOM>(Ln, st, make_float4(sF(vv), sF(nv + vv), sF(2 * nv + vv), 0.f));
    }
    return;
  }
  mark_box_tiles<GEOM>(Ln, lo2, dims2);
  if (!(fmax > 0.f)) return;
  // fixed-point box after the positions and forces (still read below)
  int* ibox = reinterpret_cast<int*>(S.sQ + 3 * nv);
  unsigned short* order = reinterpret_cast<unsigned short*>(ibox + 3 * BOX_CELLS);
  const int vol = dims2.x * dims2.y * dims2.z;
  const float Sc = fminf(33554432.0f, 8589934592.0f / (float)nv) / fmax;  // as in spread_group
  for (int i = threadIdx.x; i < 3 * vol; i += blockDim.x) ibox[i] = 0;
#pragma unroll
  for (int q = 0; q < COUPLE_PER_THREAD; ++q)
    if (l2[q] >= 0) order[atomicAdd(&R.cur[l2[q] & 31], 1)] = (unsigned short)(threadIdx.x + q * COUPLE_THREADS);
  __syncthreads();
  {
    // the order and counters for the next step's gather at these positions
    int* wmeta = reinterpret_cast<int*>(orec);
    unsigned short* widx = reinterpret_cast<unsigned short*>(orec + ORDER_META_INTS * 4);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) widx[i] = order[i];
    if (threadIdx.x < 32) {
      wmeta[threadIdx.x] = R.cnt[threadIdx.x];
      wmeta[32 + threadIdx.x] = R.start[threadIdx.x];
    }
    if (threadIdx.x == 0) wmeta[64] = R.most;
  }
  {
    const int n = R.cnt[lane], st = R.start[lane];
    for (int w = threadIdx.x >> 5; w < R.most; w += nwarps) {
      if (w >= n) continue;
      const int v = order[st + w];
      int c[3];
      float f[3];
      smem_cell(S, nv, v, o, c, f);
      const int li0 = (c[0] - 1 - lo2.x) + dims2.x * ((c[1] - 1 - lo2.y) + dims2.y * (c[2] - 1 - lo2.z));
      scatter_marker(ibox, vol, dims2, li0, f[0], f[1], f[2], sF(v) * Sc, sF(nv + v) * Sc, sF(2 * nv + v) * Sc);
    }
  }
  __syncthreads();
  flush_box<GEOM>(Ln, lo2, dims2, ibox, 1.0f / Sc);
}

template <int GEOM>
__global__ void __launch_bounds__(COUPLE_THREADS, 2)
    k_couple(LatticeDev L, float4* g_next, MarkersDev m, BodyDev* __restrict__ bodies, const int2* __restrict__ items,
             const MarkerGroup* __restrict__ groups, int4* boxes, unsigned char* orders, MeshDev mesh) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * 32];
  // items[b] = (body, group b): the items follow the group order, so the
  // group and its box are read without waiting for the item
  const int b = blockIdx.x;
  couple_membrane<GEOM>(L, g_next, m, bodies + items[b].x, groups[b], boxes + 2 * b,
                        orders + (size_t)b * couple_order_stride(mesh.nv), mesh, smem, red);
}

}  // namespace

// Shared memory of the fused kernel for a template of nv vertices: the
// largest of its regions (the velocity box with the gathered velocities and
// the gather order; the positions, forces, normals and areas; the positions
// and forces, the fixed-point box and the vertex order, then the counters).
// At 642 vertices: 107.3 KiB, two blocks per SM; templates that need more
// than COUPLE_SMEM_MAX (above ~938 vertices) take the separate kernels.
constexpr int COUPLE_SMEM_MAX = BOX_CELLS * 16 + XFER_GROUP_MAX * 16 + RESIDUE_BYTES;

size_t couple_smem(const MeshDev& mesh) {
  return (size_t)couple_counters_offset(mesh.nv, mesh.nt) + RESIDUE_BYTES;
}

size_t couple_order_bytes(const MeshDev& mesh) { return (size_t)couple_order_stride(mesh.nv); }

bool couple_fits(const MeshDev& mesh) {
  return mesh.nv >= 1 && mesh.nv <= COUPLE_PER_THREAD * COUPLE_THREADS && couple_smem(mesh) <= (size_t)COUPLE_SMEM_MAX;
}

cudaError_t couple_configure() {
  cudaError_t e = cudaSuccess;
#define CFG(k) if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, COUPLE_SMEM_MAX)
  CFG(k_couple<GEOM_PERIODIC>); CFG(k_couple<GEOM_YWALLS>); CFG(k_couple<GEOM_TUBE>);
#undef CFG
  return e;
}

void launch_couple(const LatticeDev& L, float4* g_next, const MarkersDev& m, BodyDev* bodies, const int2* items,
                   int n_items, const MarkerGroup* groups, int4* boxes, unsigned char* orders, const MeshDev& mesh,
                   cudaStream_t st) {
  if (n_items == 0) return;
  const size_t smem = couple_smem(mesh);
  switch (L.geometry) {
    case GEOM_PERIODIC:
      k_couple<GEOM_PERIODIC><<<n_items, COUPLE_THREADS, smem, st>>>(L, g_next, m, bodies, items, groups, boxes, orders, mesh);
      break;
    case GEOM_YWALLS:
      k_couple<GEOM_YWALLS><<<n_items, COUPLE_THREADS, smem, st>>>(L, g_next, m, bodies, items, groups, boxes, orders, mesh);
      break;
    default:
      k_couple<GEOM_TUBE><<<n_items, COUPLE_THREADS, smem, st>>>(L, g_next, m, bodies, items, groups, boxes, orders, mesh);
      break;
  }
}

}  // namespace ibm

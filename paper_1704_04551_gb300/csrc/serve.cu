// Serving: continuous batching of independent coupled IBM-LBM simulations on
// one GPU (ibm_lbm_server_* in include/ibm_lbm.h).
//
// Each admitted case is an ordinary ibm_lbm handle (its own lattice, markers
// and bodies in device memory, created through the server's allocator and on
// the server's stream). The server advances all of them together: one
// launch per stage for all cases, with per-case work items
//   rows   (case, fluid row)      -> collide-stream-force
//   groups (case, marker group)   -> spreading, interpolation
//   bodies (case, body)           -> marker forces
// and a device-side case table holding each case's arrays, step count and
// this step's flags (active, AA parity, dense moments on the last step). A
// chunk of steps is captured once per set of admitted cases and replayed as
// a CUDA graph; a case that reaches its step count mid-chunk is skipped for
// the rest of it. Between chunks finished cases are retired (results copied
// to host memory, device memory released) and waiting ones admitted in FIFO
// order as the memory budget and slots allow.
//
// The batched kernels call the same device bodies as the single-lattice
// kernels (lbm_cell.cuh, transfer_group.cuh, forces_body.cuh), so a case's
// result does not depend on what else is being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/ibm_lbm.h"
#include "common.cuh"
#include "forces_body.cuh"
#include "handle.h"
#include "internal.h"
#include "lbm_cell.cuh"
#include "transfer_group.cuh"

namespace ibm {
namespace {

struct CaseDev {
  LatticeDev L;  // g / flags are taken from gbuf / fbuf by parity
  float4* gbuf;
  uint8_t* fbuf;
  const RowInfo* rows;
  MarkersDev m;
  const MarkerGroup* groups;
  int4* boxes;
  BodyDev* bodies;
  MeshDev mesh;
  long long target;  // steps to run
  long long done;    // steps completed
  int active, odd, dense, ntiles, zero_F;
};

struct Item {
  int c, i;  // case, row / group / body
};

__device__ __forceinline__ LatticeDev case_lattice(const CaseDev& C) {
  LatticeDev L = C.L;
  L.g = C.gbuf;
  L.flags = C.fbuf;
  return L;
}

constexpr int SERVE_XFER_THREADS = XFER_THREADS;
constexpr int SERVE_COLLIDE_TX = 32, SERVE_COLLIDE_TY = 4;

__global__ void k_book_begin(CaseDev* cases, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  CaseDev& C = cases[t];
  C.active = C.done < C.target ? 1 : 0;
  C.odd = (int)(C.done & 1);
  C.dense = (C.done + 1 == C.target) ? 1 : 0;
}

__global__ void k_book_end(CaseDev* cases, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (cases[t].active) cases[t].done += 1;
}

// Start of a step: clear the tile flags this step's spreading marks and,
// for cases with markers outside every body, the marker forces.
__global__ void k_clear_flags(const CaseDev* cases) {
  const CaseDev& C = cases[blockIdx.x];
  if (!C.active) return;
  uint8_t* f = C.fbuf;
  for (int i = threadIdx.x; i < C.ntiles; i += blockDim.x) f[i] = 0;
  if (C.zero_F)
    for (int k = threadIdx.x; k < C.m.M; k += blockDim.x) C.m.F[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(RIGID_THREADS) k_rigid_b(const CaseDev* cases, const Item* items) {
  __shared__ double sh[6 * 32];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  rigid_block(C.m, C.bodies + it.i, sh);
}

__global__ void __launch_bounds__(MEMBRANE_THREADS, 4) k_membranes_b(const CaseDev* cases, const Item* items) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * 32];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  membrane_block(C.m, C.bodies + it.i, C.mesh, smem, red);
}

__global__ void __launch_bounds__(SERVE_XFER_THREADS, 2) k_spread_b(const CaseDev* cases, const Item* items) {
  extern __shared__ __align__(16) unsigned char ibox[];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  const LatticeDev L = case_lattice(C);
  int4* box = C.boxes + 2 * it.i;
  switch (L.geometry) {
    case GEOM_PERIODIC: spread_group<GEOM_PERIODIC>(L, C.m, C.groups[it.i], box, ibox); break;
    case GEOM_YWALLS: spread_group<GEOM_YWALLS>(L, C.m, C.groups[it.i], box, ibox); break;
    default: spread_group<GEOM_TUBE>(L, C.m, C.groups[it.i], box, ibox); break;
  }
}

__global__ void __launch_bounds__(SERVE_XFER_THREADS, 2) k_interpolate_b(const CaseDev* cases, const Item* items) {
  extern __shared__ __align__(16) unsigned char fbox[];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  const LatticeDev L = case_lattice(C);
  const int4* box = C.boxes + 2 * it.i;
  switch (L.geometry) {
    case GEOM_PERIODIC: interpolate_group<GEOM_PERIODIC>(L, C.m, C.groups[it.i], box, fbox); break;
    case GEOM_YWALLS: interpolate_group<GEOM_YWALLS>(L, C.m, C.groups[it.i], box, fbox); break;
    default: interpolate_group<GEOM_TUBE>(L, C.m, C.groups[it.i], box, fbox); break;
  }
}

// The same for chunks of fewer than LANE_MAX_GROUPS groups (four lanes per
// marker).
__global__ void __launch_bounds__(LANE_THREADS, 1) k_spread_bl(const CaseDev* cases, const Item* items) {
  extern __shared__ __align__(16) int ibox_l[];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  const LatticeDev L = case_lattice(C);
  int4* box = C.boxes + 2 * it.i;
  switch (L.geometry) {
    case GEOM_PERIODIC: spread_group_lanes<GEOM_PERIODIC>(L, C.m, C.groups[it.i], box, ibox_l); break;
    case GEOM_YWALLS: spread_group_lanes<GEOM_YWALLS>(L, C.m, C.groups[it.i], box, ibox_l); break;
    default: spread_group_lanes<GEOM_TUBE>(L, C.m, C.groups[it.i], box, ibox_l); break;
  }
}

__global__ void __launch_bounds__(LANE_THREADS, 1) k_interpolate_bl(const CaseDev* cases, const Item* items) {
  extern __shared__ __align__(16) unsigned char fbox_l[];
  const Item it = items[blockIdx.x];
  const CaseDev& C = cases[it.c];
  if (!C.active) return;
  const LatticeDev L = case_lattice(C);
  const int4* box = C.boxes + 2 * it.i;
  switch (L.geometry) {
    case GEOM_PERIODIC: interpolate_group_lanes<GEOM_PERIODIC>(L, C.m, C.groups[it.i], box, fbox_l); break;
    case GEOM_YWALLS: interpolate_group_lanes<GEOM_YWALLS>(L, C.m, C.groups[it.i], box, fbox_l); break;
    default: interpolate_group_lanes<GEOM_TUBE>(L, C.m, C.groups[it.i], box, fbox_l); break;
  }
}

// One warp per (case, row) segment of 32 cells. Cases are admitted only at
// chunk boundaries and every chunk has an even number of steps, so all
// running cases share the AA parity of a step and it is a template argument;
// rows are grouped by geometry, one launch per geometry present.
// 10 resident blocks per SM for the even step, 9 for the odd one, as for the
// single-lattice collide (64-case stream: 17,610 -> 18,150 MLUPS against 6).
template <int ODD, int GEOM>
__global__ void __launch_bounds__(SERVE_COLLIDE_TX * SERVE_COLLIDE_TY, ODD ? 9 : 10)
    k_collide_b(const CaseDev* cases, const Item* items, int n_items, int nxb) {
  const int ib = blockIdx.x / nxb, xb = blockIdx.x - ib * nxb;  // one-dimensional grid, x chunks fastest
  const int item = ib * blockDim.y + threadIdx.y;
  if (item >= n_items) return;
  const Item it = items[item];
  const CaseDev& C = cases[it.c];
  const int x = xb * blockDim.x + threadIdx.x;
  if (!C.active || x >= C.L.nx) return;
  const LatticeDev L = case_lattice(C);
  const RowInfo R = C.rows[it.i];
  // served lattices are far below 2^32 / 19 cells (checked at submission)
  if (C.dense) collide_cell<STORE_F32, ODD, GEOM, true, ODD == 1>(L, R, x);
  else collide_cell<STORE_F32, ODD, GEOM, false, ODD == 1>(L, R, x);
}

}  // namespace
}  // namespace ibm

using namespace ibm;

struct ibm_lbm_server {
  struct Case {
    uint64_t id = 0;
    int state = IBM_LBM_CASE_PENDING;
    ibm_lbm_t* h = nullptr;
    long long target = 0, steps = 0;
    size_t estimate = 0, held = 0;
    int unstable = 0;
    // inputs
    ibm_lbm_config lat{};
    std::vector<double> rho0, u0, X;
    std::vector<ibm_lbm_body> bodies;
    std::vector<int32_t> tris;
    std::vector<double> rest;
    int nv = 0, nt = 0;
    bool has_mesh = false;
    // results
    std::vector<double> rho, u, Xr, Ur;
    std::vector<ibm_lbm_body> bodies_out;
  };
  ibm_lbm_server_config cfg{};
  ibm_lbm_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<uint64_t, std::unique_ptr<Case>> cases;
  std::deque<Case*> pending;
  std::vector<Case*> running;
  uint64_t next_id = 1;
  size_t used = 0;
  // device tables
  std::vector<Alloc> mem;
  CaseDev* d_cases = nullptr;
  Item *d_rows = nullptr, *d_groups = nullptr, *d_rigid = nullptr, *d_membranes = nullptr;
  size_t cap_rows = 0, cap_groups = 0, cap_rigid = 0, cap_membranes = 0;
  int n_rows = 0, n_groups = 0, n_rigid = 0, n_membranes = 0, max_xblocks = 0;
  int geom_first[4] = {0, 0, 0, 0};  // rows of geometry g: [geom_first[g], geom_first[g + 1])
  size_t membrane_smem = 0;
  std::vector<CaseDev> h_cases;
  cudaGraphExec_t graph = nullptr;
  bool dirty = true;
  std::string err;
};

namespace {

int sfail(ibm_lbm_server_t* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

// No C++ exception crosses the C ABI (as for the handle calls): a failed
// host allocation returns E_NOMEM, any other exception E_ARG.
template <class F>
int server_guard(ibm_lbm_server_t* s, F&& body) noexcept {
  const char* msg = nullptr;
  int code = IBM_LBM_OK;
  try {
    return body();
  } catch (const std::bad_alloc&) {
    code = IBM_LBM_E_NOMEM;
    msg = "host allocation failed";
  } catch (...) {
    code = IBM_LBM_E_ARG;
    msg = "invalid size or argument (host exception)";
  }
  if (s) {
    try {
      s->err = msg;
    } catch (...) {
    }
  }
  return code;
}

#define SCUDA(s, call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return sfail((s), IBM_LBM_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

void* sdalloc(ibm_lbm_server_t* s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (s->has_alloc) p = s->alloc.alloc(bytes, s->alloc.ctx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) s->mem.push_back({p, bytes});
  return p;
}

void sdfree(ibm_lbm_server_t* s, void* p) {
  for (size_t i = 0; i < s->mem.size(); ++i)
    if (s->mem[i].p == p) {
      if (s->has_alloc) s->alloc.release(p, s->alloc.ctx);
      else cudaFree(p);
      s->mem.erase(s->mem.begin() + i);
      return;
    }
}

// Grow a device item array to hold n items.
int ensure(ibm_lbm_server_t* s, Item** buf, size_t* cap, size_t n) {
  if (n <= *cap && *buf) return IBM_LBM_OK;
  if (*buf) sdfree(s, *buf);
  size_t c = std::max<size_t>(n, 2 * *cap);
  if (c < 64) c = 64;
  *buf = (Item*)sdalloc(s, sizeof(Item) * c);
  if (!*buf) return sfail(s, IBM_LBM_E_NOMEM, "server: device allocation failed");
  *cap = c;
  return IBM_LBM_OK;
}

// Device memory a case will hold (FP32 storage), an upper bound of what the
// handle allocates: populations, wall velocities, two force-density and
// tile-flag buffers, the row table, per-marker arrays (X, U, F, stencil
// cache; reference positions of rigid markers), marker groups and boxes,
// bodies and lists, packed mesh topology, plus allocation rounding.
size_t case_estimate(const ibm_lbm_config& L, int64_t M, int n_bodies, bool rigid, int nv, int nt) {
  const size_t N = (size_t)L.nx * L.ny * L.nz;
  const size_t tiles = (size_t)((L.nx + 31) / 32) * ((L.ny + 3) / 4) * ((L.nz + 3) / 4);
  size_t b = N * (19 * 4 + 16 + 2 * 16) + 2 * tiles + (size_t)L.ny * L.nz * sizeof(RowInfo) + 1024;
  b += (size_t)M * (24 + 16 + 16 + 12 + 12 + (rigid ? 24 : 0));
  b += (size_t)(M / 256 + 64) * (sizeof(MarkerGroup) + 2 * sizeof(int4));
  b += (size_t)n_bodies * (sizeof(BodyDev) + 2 * sizeof(int));
  b += (size_t)nv * 40 + (size_t)nt * 40 + 64 * 1024;
  return b + 32 * 512;
}

void release_case(ibm_lbm_server_t* s, ibm_lbm_server::Case* c) {
  if (c->h) {
    ibm_lbm_destroy(c->h);
    c->h = nullptr;
  }
  s->used -= std::min(s->used, c->held);
  c->held = 0;
}

int admit(ibm_lbm_server_t* s) {
  while (!s->pending.empty() && (int)s->running.size() < s->cfg.max_active) {
    ibm_lbm_server::Case* c = s->pending.front();
    if (s->used + c->estimate > s->cfg.device_mem_budget) break;  // wait for memory (FIFO)
    ibm_lbm_t* h = nullptr;
    int rc = ibm_lbm_create(&c->lat, s->has_alloc ? &s->alloc : nullptr, s->stream, &h);
    if (rc == IBM_LBM_OK)
      rc = ibm_lbm_set_lattice(h, c->rho0.empty() ? nullptr : c->rho0.data(), c->u0.empty() ? nullptr : c->u0.data());
    if (rc == IBM_LBM_OK) {
      ibm_lbm_mesh mesh{c->nv, c->nt, c->tris.data(), c->rest.data()};
      const int64_t M = (int64_t)(c->X.size() / 3);
      rc = ibm_lbm_set_markers(h, c->has_mesh ? &mesh : nullptr, (int32_t)c->bodies.size(), c->bodies.data(), M,
                               c->X.data());
    }
    if (rc != IBM_LBM_OK) {
      std::string why = h ? ibm_lbm_last_error(h) : "create failed";
      if (h) ibm_lbm_destroy(h);
      if (rc == IBM_LBM_E_NOMEM) break;  // retry after retirements
      return sfail(s, rc, "server: admission failed: " + why);
    }
    c->h = h;
    c->held = ibm_lbm_device_bytes(h);
    s->used += c->held;
    c->state = IBM_LBM_CASE_RUNNING;
    c->steps = 0;
    s->running.push_back(c);
    s->pending.pop_front();
    s->dirty = true;
  }
  return IBM_LBM_OK;
}

int rebuild(ibm_lbm_server_t* s) {
  const int n = (int)s->running.size();
  std::vector<Item> rows, groups, rigid, membranes;
  std::vector<Item> rows_g[3];
  s->h_cases.assign(n, CaseDev{});
  s->max_xblocks = 0;
  s->membrane_smem = 0;
  for (int i = 0; i < n; ++i) {
    ibm_lbm_t* h = s->running[i]->h;
    CaseDev& C = s->h_cases[i];
    C.L = h->L;
    C.gbuf = h->gbuf;
    C.fbuf = h->fbuf;
    C.rows = h->rows;
    C.m = h->m;
    C.groups = h->groups;
    C.boxes = h->boxes;
    C.bodies = h->d_bodies;
    C.mesh = h->mesh;
    C.target = s->running[i]->target;
    C.done = s->running[i]->steps;
    C.ntiles = h->L.ntx * h->L.nty * h->L.ntz;
    C.zero_F = h->need_zero_F ? 1 : 0;
    const int geom = std::min(std::max(h->L.geometry, 0), 2);
    for (int r = 0; r < h->n_rows; ++r) rows_g[geom].push_back({i, r});
    if (h->m.M > 0)
      for (int g = 0; g < h->n_groups; ++g) groups.push_back({i, g});
    for (int b = 0; b < h->n_bodies; ++b) {
      const int kind = h->h_bodies[b].kind;
      if (kind == IBM_LBM_BODY_RIGID || kind == IBM_LBM_BODY_RIGID_DIRECT) rigid.push_back({i, b});
      else membranes.push_back({i, b});
    }
    if (h->n_membranes > 0)
      s->membrane_smem = std::max(s->membrane_smem, sizeof(float) * (size_t)h->mesh.work_floats);
    s->max_xblocks = std::max(s->max_xblocks, (h->L.nx + SERVE_COLLIDE_TX - 1) / SERVE_COLLIDE_TX);
  }
  for (int g = 0; g < 3; ++g) {
    s->geom_first[g] = (int)rows.size();
    rows.insert(rows.end(), rows_g[g].begin(), rows_g[g].end());
  }
  s->geom_first[3] = (int)rows.size();
  int rc;
  if ((rc = ensure(s, &s->d_rows, &s->cap_rows, rows.size()))) return rc;
  if ((rc = ensure(s, &s->d_groups, &s->cap_groups, groups.size()))) return rc;
  if ((rc = ensure(s, &s->d_rigid, &s->cap_rigid, rigid.size()))) return rc;
  if ((rc = ensure(s, &s->d_membranes, &s->cap_membranes, membranes.size()))) return rc;
  s->n_rows = (int)rows.size();
  s->n_groups = (int)groups.size();
  s->n_rigid = (int)rigid.size();
  s->n_membranes = (int)membranes.size();
  SCUDA(s, cudaMemcpyAsync(s->d_cases, s->h_cases.data(), sizeof(CaseDev) * n, cudaMemcpyHostToDevice, s->stream));
  if (!rows.empty())
    SCUDA(s, cudaMemcpyAsync(s->d_rows, rows.data(), sizeof(Item) * rows.size(), cudaMemcpyHostToDevice, s->stream));
  if (!groups.empty())
    SCUDA(s, cudaMemcpyAsync(s->d_groups, groups.data(), sizeof(Item) * groups.size(), cudaMemcpyHostToDevice,
                             s->stream));
  if (!rigid.empty())
    SCUDA(s, cudaMemcpyAsync(s->d_rigid, rigid.data(), sizeof(Item) * rigid.size(), cudaMemcpyHostToDevice, s->stream));
  if (!membranes.empty())
    SCUDA(s, cudaMemcpyAsync(s->d_membranes, membranes.data(), sizeof(Item) * membranes.size(),
                             cudaMemcpyHostToDevice, s->stream));
  if (s->membrane_smem > 48 * 1024)
    SCUDA(s, cudaFuncSetAttribute(k_membranes_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->membrane_smem));
  SCUDA(s, cudaStreamSynchronize(s->stream));
  // capture one chunk
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  const bool lanes = s->n_groups < LANE_MAX_GROUPS;
  SCUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  for (int step = 0; step < s->cfg.chunk_steps; ++step) {
    k_book_begin<<<(n + 127) / 128, 128, 0, s->stream>>>(s->d_cases, n);
    k_clear_flags<<<n, 256, 0, s->stream>>>(s->d_cases);
    if (s->n_rigid) k_rigid_b<<<s->n_rigid, RIGID_THREADS, 0, s->stream>>>(s->d_cases, s->d_rigid);
    if (s->n_membranes)
      k_membranes_b<<<s->n_membranes, MEMBRANE_THREADS, s->membrane_smem, s->stream>>>(s->d_cases, s->d_membranes);
    if (s->n_groups && lanes)
      k_spread_bl<<<s->n_groups, LANE_THREADS, SPREAD_LANES_SMEM, s->stream>>>(s->d_cases, s->d_groups);
    else if (s->n_groups)
      k_spread_b<<<s->n_groups, SERVE_XFER_THREADS, SPREAD_SMEM, s->stream>>>(s->d_cases, s->d_groups);
    for (int g = 0; g < 3; ++g) {
      const int first = s->geom_first[g], n_items = s->geom_first[g + 1] - first;
      if (n_items == 0) continue;
      const dim3 block(SERVE_COLLIDE_TX, SERVE_COLLIDE_TY);
      const int nxb = s->max_xblocks;
      const dim3 grid((unsigned)nxb * (unsigned)((n_items + SERVE_COLLIDE_TY - 1) / SERVE_COLLIDE_TY));
      const Item* items = s->d_rows + first;
      const bool odd = step & 1;
      switch (g * 2 + (odd ? 1 : 0)) {
        case 0: k_collide_b<0, GEOM_PERIODIC><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
        case 1: k_collide_b<1, GEOM_PERIODIC><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
        case 2: k_collide_b<0, GEOM_YWALLS><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
        case 3: k_collide_b<1, GEOM_YWALLS><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
        case 4: k_collide_b<0, GEOM_TUBE><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
        default: k_collide_b<1, GEOM_TUBE><<<grid, block, 0, s->stream>>>(s->d_cases, items, n_items, nxb); break;
      }
    }
    if (s->n_groups && lanes)
      k_interpolate_bl<<<s->n_groups, LANE_THREADS, INTERP_SMEM, s->stream>>>(s->d_cases, s->d_groups);
    else if (s->n_groups)
      k_interpolate_b<<<s->n_groups, SERVE_XFER_THREADS, INTERP_SMEM, s->stream>>>(s->d_cases, s->d_groups);
    k_book_end<<<(n + 127) / 128, 128, 0, s->stream>>>(s->d_cases, n);
  }
  cudaError_t ce = cudaStreamEndCapture(s->stream, &g);
  if (ce != cudaSuccess) return sfail(s, IBM_LBM_E_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return sfail(s, IBM_LBM_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
  s->dirty = false;
  return IBM_LBM_OK;
}

int retire(ibm_lbm_server_t* s, ibm_lbm_server::Case* c) {
  ibm_lbm_t* h = c->h;
  h->steps = c->steps;
  h->odd_next = (c->steps & 1) != 0;
  double diag[8];
  int rc = ibm_lbm_get_diagnostics(h, diag);
  if (rc) return sfail(s, rc, std::string("server: diagnostics: ") + ibm_lbm_last_error(h));
  c->unstable = !(diag[4] < 0.4);
  const size_t N = (size_t)h->L.N, M = (size_t)h->m.M;
  c->rho.resize(N);
  c->u.resize(3 * N);
  c->Xr.resize(3 * M);
  c->Ur.resize(3 * M);
  c->bodies_out.resize(c->bodies.size());
  if ((rc = ibm_lbm_get_fields(h, c->rho.data(), c->u.data()))) return sfail(s, rc, ibm_lbm_last_error(h));
  if (M && (rc = ibm_lbm_get_markers(h, c->Xr.data(), c->Ur.data(), nullptr))) return sfail(s, rc, ibm_lbm_last_error(h));
  if (!c->bodies.empty() &&
      (rc = ibm_lbm_get_bodies(h, c->bodies_out.data(), (int32_t)c->bodies_out.size())))
    return sfail(s, rc, ibm_lbm_last_error(h));
  release_case(s, c);
  c->state = IBM_LBM_CASE_DONE;
  // inputs are no longer needed
  std::vector<double>().swap(c->rho0);
  std::vector<double>().swap(c->u0);
  std::vector<double>().swap(c->X);
  return IBM_LBM_OK;
}

}  // namespace

extern "C" {

static int impl_ibm_lbm_server_create(const ibm_lbm_server_config* cfg, const ibm_lbm_allocator* alloc, void* stream,
                                      ibm_lbm_server_t** out) {
  if (!cfg || !out || cfg->max_active < 1 || cfg->chunk_steps < 2 || (cfg->chunk_steps & 1) ||
      cfg->device_mem_budget == 0 || (alloc && (!alloc->alloc || !alloc->release)))
    return IBM_LBM_E_ARG;
  *out = nullptr;
  auto s = new ibm_lbm_server_t();
  s->cfg = *cfg;
  if (alloc) {
    s->alloc = *alloc;
    s->has_alloc = true;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return IBM_LBM_E_CUDA;
  }
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return IBM_LBM_E_CUDA;
    }
    s->own_stream = true;
  }
  s->d_cases = (CaseDev*)sdalloc(s, sizeof(CaseDev) * (size_t)cfg->max_active);
  if (!s->d_cases || transfer_configure() != cudaSuccess) {
    cudaGetLastError();
    ibm_lbm_server_destroy(s);
    return IBM_LBM_E_NOMEM;
  }
  if (cudaFuncSetAttribute(k_spread_b, cudaFuncAttributeMaxDynamicSharedMemorySize, SPREAD_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_interpolate_b, cudaFuncAttributeMaxDynamicSharedMemorySize, INTERP_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_spread_bl, cudaFuncAttributeMaxDynamicSharedMemorySize, SPREAD_LANES_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(k_interpolate_bl, cudaFuncAttributeMaxDynamicSharedMemorySize, INTERP_SMEM) != cudaSuccess) {
    cudaGetLastError();
    ibm_lbm_server_destroy(s);
    return IBM_LBM_E_CUDA;
  }
  *out = s;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_server_destroy(ibm_lbm_server_t* s) {
  if (!s) return IBM_LBM_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (auto& kv : s->cases) release_case(s, kv.second.get());
  for (auto& a : s->mem) {
    if (s->has_alloc) s->alloc.release(a.p, s->alloc.ctx);
    else cudaFree(a.p);
  }
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_server_submit(ibm_lbm_server_t* s, const ibm_lbm_case* in, uint64_t* id) {
  if (!s || !in || !id) return sfail(s, IBM_LBM_E_ARG, "submit: null argument");
  const ibm_lbm_config& L = in->lattice;
  if (L.storage != IBM_LBM_STORE_F32) return sfail(s, IBM_LBM_E_ARG, "submit: served cases use FP32 storage");
  if (L.nx < 4 || L.ny < 4 || L.nz < 4 || 19LL * L.nx * L.ny * L.nz >= (1LL << 32) || in->n_steps < 0 ||
      in->n_markers < 0 || (in->n_markers > 0 && !in->X) || in->n_bodies < 0 || (in->n_bodies > 0 && !in->bodies))
    return sfail(s, IBM_LBM_E_ARG, "submit: invalid case");
  auto c = std::make_unique<ibm_lbm_server::Case>();
  c->id = s->next_id++;
  c->lat = L;
  c->lat.device = s->cfg.device;
  c->target = in->n_steps;
  const size_t N = (size_t)L.nx * L.ny * L.nz, M = (size_t)in->n_markers;
  if (in->rho0) c->rho0.assign(in->rho0, in->rho0 + N);
  if (in->u0) c->u0.assign(in->u0, in->u0 + 3 * N);
  if (M) c->X.assign(in->X, in->X + 3 * M);
  if (in->n_bodies) c->bodies.assign(in->bodies, in->bodies + in->n_bodies);
  bool rigid = false;
  for (auto& b : c->bodies) {
    rigid |= b.kind == IBM_LBM_BODY_RIGID || b.kind == IBM_LBM_BODY_RIGID_DIRECT;
    if (b.kind == IBM_LBM_BODY_FILAMENT)
      return sfail(s, IBM_LBM_E_ARG, "submit: served cases hold membranes, rigid bodies and tracers");
  }
  if (in->mesh) {
    if (!in->mesh->tris || !in->mesh->rest_X || in->mesh->n_vertices < 4 || in->mesh->n_triangles < 4)
      return sfail(s, IBM_LBM_E_ARG, "submit: invalid mesh");
    c->has_mesh = true;
    c->nv = in->mesh->n_vertices;
    c->nt = in->mesh->n_triangles;
    c->tris.assign(in->mesh->tris, in->mesh->tris + 3 * (size_t)c->nt);
    c->rest.assign(in->mesh->rest_X, in->mesh->rest_X + 3 * (size_t)c->nv);
  }
  c->estimate = case_estimate(L, in->n_markers, in->n_bodies, rigid, c->nv, c->nt);
  if (c->estimate > s->cfg.device_mem_budget) return sfail(s, IBM_LBM_E_ARG, "submit: case exceeds the memory budget");
  *id = c->id;
  s->pending.push_back(c.get());
  s->cases[c->id] = std::move(c);
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_server_advance(ibm_lbm_server_t* s, int32_t* n_running, int32_t* n_pending, int32_t* n_done) {
  if (!s) return IBM_LBM_E_ARG;
  int rc = admit(s);
  if (rc) return rc;
  int status = IBM_LBM_OK;
  if (!s->running.empty()) {
    if (s->dirty && (rc = rebuild(s))) return rc;
    SCUDA(s, cudaGraphLaunch(s->graph, s->stream));
    const int n = (int)s->running.size();
    s->h_cases.resize(n);
    SCUDA(s, cudaMemcpyAsync(s->h_cases.data(), s->d_cases, sizeof(CaseDev) * n, cudaMemcpyDeviceToHost, s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    std::vector<ibm_lbm_server::Case*> still;
    for (int i = 0; i < n; ++i) {
      ibm_lbm_server::Case* c = s->running[i];
      c->steps = s->h_cases[i].done;
      if (c->steps >= c->target) {
        if ((rc = retire(s, c))) return rc;
        if (c->unstable) status = IBM_LBM_E_UNSTABLE;
        s->dirty = true;
      } else {
        still.push_back(c);
      }
    }
    s->running.swap(still);
    if ((rc = admit(s))) return rc;
  }
  int done = 0;
  for (auto& kv : s->cases) done += kv.second->state == IBM_LBM_CASE_DONE;
  if (n_running) *n_running = (int32_t)s->running.size();
  if (n_pending) *n_pending = (int32_t)s->pending.size();
  if (n_done) *n_done = done;
  if (status) s->err = "a retired case failed its conservation check";
  return status;
}

static int impl_ibm_lbm_server_poll(ibm_lbm_server_t* s, uint64_t id, int32_t* state, int64_t* steps_done) {
  if (!s) return IBM_LBM_E_ARG;
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return sfail(s, IBM_LBM_E_ARG, "poll: unknown case");
  if (state) *state = it->second->state;
  if (steps_done) *steps_done = it->second->steps;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_server_result(ibm_lbm_server_t* s, uint64_t id, double* rho, double* u, double* X, double* U,
                                      ibm_lbm_body* bodies, int32_t n_bodies) {
  if (!s) return IBM_LBM_E_ARG;
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return sfail(s, IBM_LBM_E_ARG, "result: unknown case");
  ibm_lbm_server::Case* c = it->second.get();
  if (c->state != IBM_LBM_CASE_DONE) return sfail(s, IBM_LBM_E_STATE, "result: case not finished");
  if (bodies && n_bodies != (int32_t)c->bodies_out.size()) return sfail(s, IBM_LBM_E_ARG, "result: body count");
  if (rho) std::memcpy(rho, c->rho.data(), sizeof(double) * c->rho.size());
  if (u) std::memcpy(u, c->u.data(), sizeof(double) * c->u.size());
  if (X) std::memcpy(X, c->Xr.data(), sizeof(double) * c->Xr.size());
  if (U) std::memcpy(U, c->Ur.data(), sizeof(double) * c->Ur.size());
  if (bodies && n_bodies) std::memcpy(bodies, c->bodies_out.data(), sizeof(ibm_lbm_body) * n_bodies);
  s->cases.erase(it);
  return IBM_LBM_OK;
}

const char* ibm_lbm_server_last_error(const ibm_lbm_server_t* s) { return s ? s->err.c_str() : "null server"; }


int ibm_lbm_server_create(const ibm_lbm_server_config* cfg, const ibm_lbm_allocator* alloc, void* stream,
                          ibm_lbm_server_t** out) {
  return server_guard(nullptr, [&]() -> int { return impl_ibm_lbm_server_create(cfg, alloc, stream, out); });
}

int ibm_lbm_server_destroy(ibm_lbm_server_t* s) {
  return server_guard(s, [&]() -> int { return impl_ibm_lbm_server_destroy(s); });
}

int ibm_lbm_server_submit(ibm_lbm_server_t* s, const ibm_lbm_case* in, uint64_t* id) {
  return server_guard(s, [&]() -> int { return impl_ibm_lbm_server_submit(s, in, id); });
}

int ibm_lbm_server_advance(ibm_lbm_server_t* s, int32_t* n_running, int32_t* n_pending, int32_t* n_done) {
  return server_guard(s, [&]() -> int { return impl_ibm_lbm_server_advance(s, n_running, n_pending, n_done); });
}

int ibm_lbm_server_poll(ibm_lbm_server_t* s, uint64_t id, int32_t* state, int64_t* steps_done) {
  return server_guard(s, [&]() -> int { return impl_ibm_lbm_server_poll(s, id, state, steps_done); });
}

int ibm_lbm_server_result(ibm_lbm_server_t* s, uint64_t id, double* rho, double* u, double* X, double* U,
                          ibm_lbm_body* bodies, int32_t n_bodies) {
  return server_guard(s, [&]() -> int { return impl_ibm_lbm_server_result(s, id, rho, u, X, U, bodies, n_bodies); });
}
}  // extern "C"

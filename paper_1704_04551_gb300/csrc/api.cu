// C ABI of the coupled IBM-LBM step (include/ibm_lbm.h): handle lifetime,
// device memory, host<->device conversion, validation, and the step loop
// (captured into CUDA graphs: one graph per 16 steps, plus single steps).
#include <cuda_runtime.h>

#include <unistd.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ibm_lbm.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"
#include "transfer_group.cuh"

using namespace ibm;

static_assert(BODY_GROUP <= XFER_GROUP_MAX && TRACER_GROUP <= XFER_GROUP_MAX,
              "transfer groups must fit the shared-memory marker records");

namespace {

int fail(ibm_lbm_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

// No C++ exception crosses the C ABI: every entry point runs its body under
// this guard; a failed host allocation returns E_NOMEM, any other exception
// (e.g. a size the standard containers reject) E_ARG.
template <class F>
int abi_guard(ibm_lbm_t* h, F&& body) noexcept {
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
  if (h) {
    try {
      h->err = msg;
    } catch (...) {
    }
  }
  return code;
}

#define CUDA_TRY(h, call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((h), IBM_LBM_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_));   \
  } while (0)

void* dalloc(ibm_lbm_t* h, std::vector<Alloc>& pool, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(bytes, h->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    pool.push_back({p, bytes});
    h->bytes += bytes;
  }
  return p;
}

// Take the page faults of a large host buffer on several threads: one byte
// per page is written (an output that is about to be overwritten) or read
// (an input), so that a freshly allocated buffer is mapped in parallel
// before a copy, which would fault its pages one by one.
void touch_pages(const void* p, size_t bytes, bool write) {
  if (!p || bytes < ((size_t)16 << 20)) return;
  const long pg = sysconf(_SC_PAGESIZE);
  const size_t page = pg > 0 ? (size_t)pg : 4096;
  const unsigned nt = std::min(8u, std::max(1u, std::thread::hardware_concurrency()));
  const size_t chunk = (bytes / nt + page - 1) / page * page;
  auto touch = [p, page, write](size_t b, size_t e) {
    if (write) {
      volatile char* q = static_cast<volatile char*>(const_cast<void*>(p));
      for (size_t o = b; o < e; o += page) q[o] = 0;
    } else {
      const volatile char* q = static_cast<const volatile char*>(p);
      char sink = 0;
      for (size_t o = b; o < e; o += page) sink ^= q[o];
      (void)sink;
    }
  };
  std::vector<std::thread> th;
  size_t done = 0;  // [0, done) is handed to threads
  try {
    for (unsigned t = 0; t < nt; ++t) {
      const size_t b = t * chunk, e = std::min(bytes, b + chunk);
      if (b >= e) break;
      th.emplace_back(touch, b, e);
      done = e;
    }
  } catch (...) {
    // no more threads: the calling thread takes the rest (an optimisation only)
  }
  touch(done, bytes);
  for (auto& x : th) x.join();
}

void release_pool(ibm_lbm_t* h, std::vector<Alloc>& pool) {
  for (auto& a : pool) {
    if (h->has_alloc) h->alloc.release(a.p, h->alloc.ctx);
    else cudaFree(a.p);
    h->bytes -= a.bytes;
  }
  pool.clear();
}

void drop_graphs(ibm_lbm_t* h) {
  if (h->g_chunk) cudaGraphExecDestroy(h->g_chunk);
  h->g_chunk = nullptr;
  for (auto& row : h->g_single)
    for (auto& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto& g : h->g_fused) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

int tiles(const LatticeDev& L) { return L.ntx * L.nty * L.ntz; }

// Lattice view for a step (the AA parity is a kernel template argument, the
// force density and its flags are single buffers).
LatticeDev lat(const ibm_lbm_t* h, bool odd) {
  (void)odd;
  return h->L;
}

// Marker forces: each body's own forces (membranes, rigid tethers,
// filaments), then the Morse excluded volume between bodies.
void enqueue_forces(ibm_lbm_t* h, cudaStream_t st) {
  if (h->m.M == 0) return;
  if (h->need_zero_F) cudaMemsetAsync(h->m.F, 0, sizeof(float4) * (size_t)h->m.M, st);
  launch_forces(h->m, h->d_bodies, h->membrane_list, h->n_membranes, h->rigid_list, h->n_rigids, h->mesh, st);
  launch_filaments(h->m, h->d_bodies, h->filament_list, h->n_filaments, st);
  if (h->morse_rc > 0.0 && h->morse_ready)
    launch_morse(h->morse, h->m, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->cfg.geometry, st);
}

// One coupled step on the handle's stream (also used under capture).
void enqueue_step(ibm_lbm_t* h, bool odd, bool dense) {
  cudaStream_t st = h->stream;
  const LatticeDev L = lat(h, odd);
  cudaMemsetAsync(L.flags, 0, (size_t)tiles(L), st);
  if (h->m.M > 0) {
    enqueue_forces(h, st);
    launch_spread(L, h->m, h->groups, h->n_groups, h->boxes, st);
  }
  launch_collide(L, h->rows, h->n_rows, h->cfg.storage, odd, dense, st);
  if (h->m.M > 0) launch_interpolate(L, h->m, h->groups, h->n_groups, h->boxes, st);
}

// One step with an event before each stage and after the last.
void enqueue_timed_step(ibm_lbm_t* h, bool odd, bool dense) {
  cudaStream_t st = h->stream;
  const size_t base = 5 * h->timed_steps;
  const bool rec = base + 5 <= h->events.size();
  auto mark = [&](int k) {
    if (rec) cudaEventRecord(h->events[base + k], st);
  };
  const LatticeDev L = lat(h, odd);
  cudaMemsetAsync(L.flags, 0, (size_t)tiles(L), st);
  mark(0);
  enqueue_forces(h, st);
  mark(1);
  if (h->m.M > 0) launch_spread(L, h->m, h->groups, h->n_groups, h->boxes, st);
  mark(2);
  launch_collide(L, h->rows, h->n_rows, h->cfg.storage, odd, dense, st);
  mark(3);
  if (h->m.M > 0) launch_interpolate(L, h->m, h->groups, h->n_groups, h->boxes, st);
  mark(4);
  if (rec) {
    h->timed_odd.push_back(odd ? 1 : 0);
    h->timed_fused.push_back(0);
    h->timed_steps++;
  }
}

int capture(ibm_lbm_t* h, cudaGraphExec_t* out, int n, bool odd0, bool dense_last) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  bool odd = odd0;
  for (int s = 0; s < n; ++s) {
    enqueue_step(h, odd, dense_last && s == n - 1);
    odd = !odd;
  }
  CUDA_TRY(h, cudaStreamEndCapture(h->stream, &g));
  cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, IBM_LBM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return IBM_LBM_OK;
}

// The fused path: n (even) coupled steps starting at an even AA step. The
// first step's forces and spreading run as separate kernels into the first
// force-density buffer; then every step is the collision (reading the
// buffer of its parity) followed by the fused kernel, which interpolates and
// advects, computes the forces at the new positions and spreads them into
// the other buffer; the last step's interpolation runs alone. The tile flags
// are cleared between a collision and the spreading that follows it.
bool fused_applies(const ibm_lbm_t* h) {
  return h->n_couple > 0 && (!h->timing || h->timing_fused) && !(h->morse_rc > 0.0) && h->gbuf2 != nullptr;
}

// With timed, the steps that launch the fused kernel record the events
// around the collision and around the tile-flag clear and the fused kernel
// (the forces and spreading slots of such a step are not read); the first
// step's forces and spreading and the last step's interpolation lie outside
// the timed intervals.
void enqueue_fused_chunk(ibm_lbm_t* h, int n, bool timed) {
  cudaStream_t st = h->stream;
  LatticeDev L0 = h->L;
  L0.g = h->gbuf;
  cudaMemsetAsync(L0.flags, 0, (size_t)tiles(L0), st);
  enqueue_forces(h, st);
  launch_spread(L0, h->m, h->groups, h->n_groups, h->boxes, st);
  for (int s = 0; s < n; ++s) {
    const size_t base = 5 * h->timed_steps;
    const bool rec = timed && s + 1 < n && base + 5 <= h->events.size();
    auto mark = [&](int k) {
      if (rec) cudaEventRecord(h->events[base + k], st);
    };
    LatticeDev Ls = h->L;
    Ls.g = (s & 1) ? h->gbuf2 : h->gbuf;
    mark(2);
    launch_collide(Ls, h->rows, h->n_rows, h->cfg.storage, (s & 1) != 0, false, st);
    mark(3);
    if (s + 1 < n) {
      cudaMemsetAsync(Ls.flags, 0, (size_t)tiles(Ls), st);
      launch_couple(Ls, (s & 1) ? h->gbuf : h->gbuf2, h->m, h->d_bodies, h->couple_items, h->n_couple, h->groups,
                    h->boxes, h->couple_order, h->mesh, st);
    } else {
      launch_interpolate(Ls, h->m, h->groups, h->n_groups, h->boxes, st);
    }
    mark(4);
    if (rec) {
      h->timed_odd.push_back((s & 1) ? 1 : 0);
      h->timed_fused.push_back(1);
      h->timed_steps++;
    }
  }
}

int capture_fused(ibm_lbm_t* h, cudaGraphExec_t* out, int n) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_fused_chunk(h, n, false);
  CUDA_TRY(h, cudaStreamEndCapture(h->stream, &g));
  cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, IBM_LBM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return IBM_LBM_OK;
}

int enqueue_diagnostics(ibm_lbm_t* h) {
  cudaStream_t st = h->stream;
  CUDA_TRY(h, cudaMemsetAsync(h->d_diag, 0, 8 * sizeof(double), st));
  CUDA_TRY(h, cudaMemsetAsync(h->d_umax, 0, sizeof(unsigned), st));
  launch_diagnostics(h->L, h->rows, h->n_rows, h->d_diag, h->d_umax, st);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(h->h_diag, h->d_diag, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_umax, h->d_umax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_status, h->L.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  h->diag_pending = true;
  return IBM_LBM_OK;
}

int finish_diagnostics(ibm_lbm_t* h) {
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (!h->diag_pending) return IBM_LBM_OK;
  h->diag_pending = false;
  float umax2;
  std::memcpy(&umax2, h->h_umax, sizeof(float));
  if (*h->h_status != 0 || !std::isfinite(umax2) || umax2 > 0.16f) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "unstable: non-finite moments or |u| > 0.4 (max |u|^2 = %g) after %lld steps",
                  (double)umax2, h->steps);
    return fail(h, IBM_LBM_E_UNSTABLE, buf);
  }
  return IBM_LBM_OK;
}

int enqueue_steps(ibm_lbm_t* h, int64_t n) {
  if (n < 0) return fail(h, IBM_LBM_E_ARG, "n_steps < 0");
  if (n == 0) return IBM_LBM_OK;
  h->boxes_valid = false;  // the last interpolation moves the markers
  int64_t left = n;
  if (h->n_couple > 0 && !h->gbuf2 && (h->timing ? h->timing_fused && left > 2 : left > CHUNK)) {
    // second force-density buffer of the fused path, zero like the first
    h->gbuf2 = (float4*)dalloc(h, h->lattice_mem, sizeof(float4) * (size_t)h->L.N);
    if (h->gbuf2) CUDA_TRY(h, cudaMemsetAsync(h->gbuf2, 0, sizeof(float4) * (size_t)h->L.N, h->stream));
  }
  if (h->timing) {
    // with timing_fused, a handle on the fused path times only its fused
    // steps; every other handle is timed stage by stage
    const bool fused = h->timing_fused && fused_applies(h);
    while (left > 0) {
      if (fused && !h->odd_next && left > 2) {
        // the fused path with direct launches; the last step stays separate
        // (it writes the velocity of every cell)
        const int m = (int)std::min<int64_t>(left - 1, 1 << 22);
        enqueue_fused_chunk(h, m, true);
        left -= m;
        h->steps += m;
        if (m & 1) h->odd_next = !h->odd_next;
        continue;
      }
      if (fused) enqueue_step(h, h->odd_next, left == 1);
      else enqueue_timed_step(h, h->odd_next, left == 1);
      --left;
      h->steps += 1;
      h->odd_next = !h->odd_next;
    }
    CUDA_TRY(h, cudaGetLastError());
    return enqueue_diagnostics(h);
  }
  while (left > 0) {
    if (fused_applies(h) && !h->odd_next && left > CHUNK) {
      const int which = left > FUSED_LONG ? 0 : 1;
      const int n = which == 0 ? FUSED_LONG : CHUNK;
      if (!h->g_fused[which]) {
        int rc = capture_fused(h, &h->g_fused[which], n);
        if (rc) return rc;
      }
      CUDA_TRY(h, cudaGraphLaunch(h->g_fused[which], h->stream));
      left -= n;
      h->steps += n;
    } else if (!h->odd_next && left > CHUNK) {
      if (!h->g_chunk) {
        int rc = capture(h, &h->g_chunk, CHUNK, false, false);
        if (rc) return rc;
      }
      CUDA_TRY(h, cudaGraphLaunch(h->g_chunk, h->stream));
      left -= CHUNK;
      h->steps += CHUNK;
    } else {
      const int odd = h->odd_next ? 1 : 0, dense = (left == 1) ? 1 : 0;
      if (!h->g_single[odd][dense]) {
        int rc = capture(h, &h->g_single[odd][dense], 1, odd, dense);
        if (rc) return rc;
      }
      CUDA_TRY(h, cudaGraphLaunch(h->g_single[odd][dense], h->stream));
      left -= 1;
      h->steps += 1;
      h->odd_next = !h->odd_next;
    }
  }
  return enqueue_diagnostics(h);
}

// ---- membrane template: edges and rest state (FP64) --------------------------
struct HostMesh {
  std::vector<int4> edges;
  std::vector<int2> edge_tris;
  std::vector<float4> edge_rest;
  std::vector<int> v_edge_start, v_edge, v_tri_start, v_tri;
  std::vector<int4> tris;
  std::vector<float> area0;
  double A0 = 0, V0 = 0;
};

struct V3 {
  double x, y, z;
};
V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 crs(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double dt3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Orders items (triangles or edges) so that, in each run of 32 consecutive
// items (one warp of the membrane force kernel), the vertices (and
// triangles) an item reads and accumulates into in each of its roles differ
// modulo 32: the warp's shared-memory accesses for one role then fall in
// distinct banks. Greedy: each run takes the first remaining items whose
// residues are all still free; a run that finds none completes with the
// items of fewest clashes. Only the order changes, not the items.
template <int R>
std::vector<int> bank_order(const std::vector<std::array<int, R>>& keys) {
  const int n = (int)keys.size();
  std::vector<int> order;
  order.reserve(n);
  std::vector<char> taken(n, 0);
  int left = n;
  while (left > 0) {
    uint32_t used[R] = {};
    int in_run = 0;
    for (int pass = 0; pass < 2 && in_run < 32 && in_run < left; ++pass) {
      for (int i = 0; i < n && in_run < 32 && in_run < left; ++i) {
        if (taken[i]) continue;
        int clash = 0;
        for (int r = 0; r < R; ++r) clash += (used[r] >> (keys[i][r] & 31)) & 1u;
        if (pass == 0 && clash) continue;
        taken[i] = 1;
        order.push_back(i);
        for (int r = 0; r < R; ++r) used[r] |= 1u << (keys[i][r] & 31);
        ++in_run;
      }
    }
    left -= in_run;
  }
  return order;
}

void order_for_banks(HostMesh& m) {
  // triangles: their three vertices
  std::vector<std::array<int, 3>> tk(m.tris.size());
  for (size_t t = 0; t < m.tris.size(); ++t) tk[t] = {m.tris[t].x, m.tris[t].y, m.tris[t].z};
  const std::vector<int> to = bank_order<3>(tk);
  std::vector<int> new_of_t(m.tris.size());
  std::vector<int4> tris(m.tris.size());
  for (size_t i = 0; i < to.size(); ++i) {
    tris[i] = m.tris[to[i]];
    new_of_t[to[i]] = (int)i;
  }
  m.tris.swap(tris);
  for (auto& et : m.edge_tris) et = make_int2(new_of_t[et.x], new_of_t[et.y]);
  // edges: their four vertices and two triangles
  std::vector<std::array<int, 6>> ek(m.edges.size());
  for (size_t e = 0; e < m.edges.size(); ++e)
    ek[e] = {m.edges[e].x, m.edges[e].y, m.edges[e].z, m.edges[e].w, m.edge_tris[e].x, m.edge_tris[e].y};
  const std::vector<int> eo = bank_order<6>(ek);
  std::vector<int4> edges(m.edges.size());
  std::vector<int2> et(m.edges.size());
  for (size_t i = 0; i < eo.size(); ++i) {
    edges[i] = m.edges[eo[i]];
    et[i] = m.edge_tris[eo[i]];
  }
  m.edges.swap(edges);
  m.edge_tris.swap(et);
}

bool build_mesh(const ibm_lbm_mesh* mesh, HostMesh& out, std::string& why) {
  const int nv = mesh->n_vertices, nt = mesh->n_triangles;
  if (nv < 4 || nv > MAX_MESH_VERTICES || nt < 4 || !mesh->tris || !mesh->rest_X) {
    why = "mesh: need 4 <= n_vertices <= 4096, n_triangles >= 4 and both arrays";
    return false;
  }
  auto P = [&](int v) { return V3{mesh->rest_X[v], mesh->rest_X[nv + v], mesh->rest_X[2 * nv + v]}; };
  std::unordered_map<uint64_t, int> emap;
  out.edges.clear();
  out.edge_tris.clear();
  out.tris.resize(nt);
  for (int t = 0; t < nt; ++t) {
    int v[3] = {mesh->tris[3 * t], mesh->tris[3 * t + 1], mesh->tris[3 * t + 2]};
    for (int s = 0; s < 3; ++s)
      if (v[s] < 0 || v[s] >= nv) {
        why = "mesh: triangle vertex index out of range";
        return false;
      }
    out.tris[t] = make_int4(v[0], v[1], v[2], 0);
    for (int s = 0; s < 3; ++s) {
      const int a = v[s], b = v[(s + 1) % 3], c = v[(s + 2) % 3];
      const uint64_t key = ((uint64_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
      auto it = emap.find(key);
      if (it == emap.end()) {
        emap.emplace(key, (int)out.edges.size());
        out.edges.push_back(make_int4(a, b, c, -1));
        out.edge_tris.push_back(make_int2(t, -1));
      } else {
        int4& e = out.edges[it->second];
        if (e.w >= 0 || e.x != b || e.y != a) {
          why = "mesh: not a closed, consistently oriented 2-manifold";
          return false;
        }
        e.w = c;
        out.edge_tris[it->second].y = t;
      }
    }
  }
  for (auto& e : out.edges)
    if (e.w < 0) {
      why = "mesh: open boundary edge";
      return false;
    }
  order_for_banks(out);
  out.edge_rest.resize(out.edges.size());
  for (size_t i = 0; i < out.edges.size(); ++i) {
    const int4 e = out.edges[i];
    V3 a = P(e.x), b = P(e.y), c = P(e.z), d = P(e.w);
    V3 ev = sub(b, a);
    V3 n1 = crs(ev, sub(c, a)), n2 = crs(sub(a, b), sub(d, b));
    const double L = std::sqrt(dt3(ev, ev));
    const double th = std::atan2(dt3(crs(n1, n2), ev) / L, dt3(n1, n2));
    out.edge_rest[i] = make_float4((float)L, (float)std::cos(th), (float)std::sin(th), 0.f);
  }
  out.area0.resize(nt);
  out.A0 = out.V0 = 0;
  for (int t = 0; t < nt; ++t) {
    V3 p0 = P(out.tris[t].x), p1 = P(out.tris[t].y), p2 = P(out.tris[t].z);
    V3 N = crs(sub(p1, p0), sub(p2, p0));
    const double A = 0.5 * std::sqrt(dt3(N, N));
    out.area0[t] = (float)A;
    out.A0 += A;
    out.V0 += dt3(p0, crs(p1, p2)) / 6.0;
  }
  if (!(out.V0 > 0)) {
    why = "mesh: non-positive rest volume (triangles must be counter-clockwise seen from outside)";
    return false;
  }
  // per-vertex lists of (edge, role) and (triangle, slot), CSR
  std::vector<std::vector<int>> ve(nv), vt(nv);
  for (size_t e = 0; e < out.edges.size(); ++e) {
    const int4 E = out.edges[e];
    ve[E.x].push_back((int)(e << 2) | 0);
    ve[E.y].push_back((int)(e << 2) | 1);
    ve[E.z].push_back((int)(e << 2) | 2);
    ve[E.w].push_back((int)(e << 2) | 3);
  }
  for (int t = 0; t < nt; ++t) {
    vt[out.tris[t].x].push_back((t << 2) | 0);
    vt[out.tris[t].y].push_back((t << 2) | 1);
    vt[out.tris[t].z].push_back((t << 2) | 2);
  }
  out.v_edge_start.assign(1, 0);
  out.v_tri_start.assign(1, 0);
  out.v_edge.clear();
  out.v_tri.clear();
  for (int v = 0; v < nv; ++v) {
    out.v_edge.insert(out.v_edge.end(), ve[v].begin(), ve[v].end());
    out.v_tri.insert(out.v_tri.end(), vt[v].begin(), vt[v].end());
    out.v_edge_start.push_back((int)out.v_edge.size());
    out.v_tri_start.push_back((int)out.v_tri.size());
  }
  return true;
}

template <typename T>
int upload(ibm_lbm_t* h, std::vector<Alloc>& pool, T** dst, const T* src, size_t count) {
  *dst = static_cast<T*>(dalloc(h, pool, sizeof(T) * count));
  if (!*dst) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
  if (count) CUDA_TRY(h, cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
  return IBM_LBM_OK;
}

void quat_matrix(const double q[4], double R[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

bool fluid_yz(const LatticeDev& L, int y, int z) {
  if (L.geometry == GEOM_YWALLS) return y >= 0 && y < L.ny;
  if (L.geometry == GEOM_TUBE) {
    if (y < 0 || y >= L.ny || z < 0 || z >= L.nz) return false;
    const float dy = (float)y - L.yc, dz = (float)z - L.zc;
    return !(dy * dy + dz * dz > L.R2);
  }
  return true;
}

std::vector<RowInfo> build_rows(const LatticeDev& L) {
  std::vector<RowInfo> rows;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      if (!fluid_yz(L, y, z)) continue;
      RowInfo R{};
      R.base = nx * (y + ny * z);
      R.y = y;
      R.trow = L.ntx * ((y >> TILE_Y_SHIFT) + L.nty * (z >> TILE_Z_SHIFT));
      R.oyp = (y == ny - 1) ? -(ny - 1) * nx : nx;
      R.oym = (y == 0) ? (ny - 1) * nx : -nx;
      R.ozp = (z == nz - 1) ? -(nz - 1) * nx * ny : nx * ny;
      R.ozm = (z == 0) ? (nz - 1) * nx * ny : -nx * ny;
      int mask = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int yy = y + dy, zz = z + dz;
          if (L.geometry == GEOM_PERIODIC) continue;
          if (L.geometry == GEOM_YWALLS) zz = (zz + nz) % nz;
          if (!fluid_yz(L, yy, zz)) mask |= 1 << ((dy + 1) * 3 + (dz + 1));
        }
      R.smask = mask;
      rows.push_back(R);
    }
  return rows;
}

// Cell-list buffers of the Morse interaction for the current markers:
// bins at least rc wide on every axis, at most morse_max_bins() of them.
int prepare_morse(ibm_lbm_t* h) {
  release_pool(h, h->morse_mem);
  h->morse_ready = false;
  const int M = h->m.M;
  const double rc = h->morse_rc;
  // neighbour lists: cutoff rc + skin, rebuilt after a move of skin / 2
  const double skin = 0.3 * rc;
  constexpr int kListCap = 48;
  const int n[3] = {h->cfg.nx, h->cfg.ny, h->cfg.nz};
  int nb[3];
  for (int a = 0; a < 3; ++a) nb[a] = std::max(1, (int)std::floor(n[a] / (rc + skin)));
  while ((long long)nb[0] * nb[1] * nb[2] > morse_max_bins()) {
    const int a = nb[0] >= nb[1] && nb[0] >= nb[2] ? 0 : (nb[1] >= nb[2] ? 1 : 2);
    nb[a] = std::max(1, nb[a] / 2);
  }
  MorseDev& P = h->morse;
  P = MorseDev{};
  P.D0 = (float)h->morse_D0;
  P.alpha = (float)h->morse_alpha;
  P.r0 = (float)h->morse_r0;
  P.rc2 = (float)(rc * rc);
  P.rl2 = (float)((rc + skin) * (rc + skin));
  P.half_skin2 = (float)(0.25 * skin * skin);
  P.cap = kListCap;
  for (int a = 0; a < 3; ++a) {
    P.nb[a] = nb[a];
    P.inv_bs[a] = (float)nb[a] / (float)n[a];
  }
  P.n_bins = nb[0] * nb[1] * nb[2];
  P.owner = h->owner;
  const size_t Mx = (size_t)std::max(M, 1);
  P.count = (int*)dalloc(h, h->morse_mem, sizeof(int) * P.n_bins);
  P.start = (int*)dalloc(h, h->morse_mem, sizeof(int) * ((size_t)P.n_bins + 1));
  P.block_sum = (int*)dalloc(h, h->morse_mem, sizeof(int) * (size_t)morse_scan_tiles(P.n_bins));
  P.bin_of = (int*)dalloc(h, h->morse_mem, sizeof(int) * Mx);
  P.rank = (int*)dalloc(h, h->morse_mem, sizeof(int) * Mx);
  P.sorted = (float4*)dalloc(h, h->morse_mem, sizeof(float4) * Mx);
  P.sorted_id = (int*)dalloc(h, h->morse_mem, sizeof(int) * Mx);
  P.bin_owner = (int*)dalloc(h, h->morse_mem, sizeof(int) * P.n_bins);
  P.ref = (float4*)dalloc(h, h->morse_mem, sizeof(float4) * Mx);
  P.cur = (float4*)dalloc(h, h->morse_mem, sizeof(float4) * Mx);
  P.n_nbr = (int*)dalloc(h, h->morse_mem, sizeof(int) * Mx);
  P.nbr = (int*)dalloc(h, h->morse_mem, sizeof(int) * Mx * kListCap);
  P.flags = (int*)dalloc(h, h->morse_mem, sizeof(int) * 2);
  if (!P.count || !P.start || !P.block_sum || !P.bin_of || !P.rank || !P.sorted || !P.sorted_id || !P.bin_owner ||
      !P.ref || !P.cur || !P.n_nbr || !P.nbr || !P.flags)
    return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
  const int flags0[2] = {1, 0};  // build the lists at the first step
  CUDA_TRY(h, cudaMemcpy(P.flags, flags0, sizeof(flags0), cudaMemcpyHostToDevice));
  CUDA_TRY(h, cudaMemset(P.ref, 0, sizeof(float4) * Mx));
  CUDA_TRY(h, cudaMemset(P.n_nbr, 0, sizeof(int) * Mx));
  CUDA_TRY(h, cudaMemset(P.count, 0, sizeof(int) * P.n_bins));
  CUDA_TRY(h, cudaMemset(P.bin_owner, 0xff, sizeof(int) * P.n_bins));
  CUDA_TRY(h, cudaMemset(P.start, 0, sizeof(int) * ((size_t)P.n_bins + 1)));
  h->morse_ready = true;
  return IBM_LBM_OK;
}

}  // namespace

extern "C" {

const char* ibm_lbm_version(void) { return "ibm_lbm 0.1 (sm_103a)"; }

const char* ibm_lbm_last_error(const ibm_lbm_t* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

void* ibm_lbm_stream(ibm_lbm_t* h) { return h ? (void*)h->stream : nullptr; }

size_t ibm_lbm_device_bytes(const ibm_lbm_t* h) { return h ? h->bytes : 0; }

static int impl_ibm_lbm_create(const ibm_lbm_config* cfg, const ibm_lbm_allocator* alloc, void* stream, ibm_lbm_t** out) {
  if (!cfg || !out) return IBM_LBM_E_ARG;
  *out = nullptr;
  const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (cfg->nx < 4 || cfg->ny < 4 || cfg->nz < 4 || N >= (1LL << 31)) return IBM_LBM_E_ARG;
  if (!(cfg->tau > 0.5) || cfg->geometry < 0 || cfg->geometry > 2 || cfg->storage < 0 || cfg->storage > 2)
    return IBM_LBM_E_ARG;
  if (cfg->geometry == 2 && !(cfg->tube_radius > 0)) return IBM_LBM_E_ARG;
  if (alloc && (!alloc->alloc || !alloc->release)) return IBM_LBM_E_ARG;
  ibm_lbm_t* h = new ibm_lbm_t();
  h->cfg = *cfg;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  auto bail = [&](int code) {
    ibm_lbm_destroy(h);
    return code;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(IBM_LBM_E_CUDA);
  }
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(IBM_LBM_E_CUDA);
    h->own_stream = true;
  }
  LatticeDev& L = h->L;
  L.nx = cfg->nx; L.ny = cfg->ny; L.nz = cfg->nz; L.N = (int)N;
  L.geometry = cfg->geometry;
  L.omega = (float)(1.0 / cfg->tau);
  L.guo_pre = (float)(1.0 - 0.5 / cfg->tau);
  L.wall_u0 = (float)cfg->wall_u[0]; L.wall_u1 = (float)cfg->wall_u[1];
  L.yc = 0.5f * (float)(cfg->ny - 1); L.zc = 0.5f * (float)(cfg->nz - 1);
  L.R2 = (float)(cfg->tube_radius * cfg->tube_radius);
  L.g0x = (float)cfg->body_force[0]; L.g0y = (float)cfg->body_force[1]; L.g0z = (float)cfg->body_force[2];
  L.ntx = (cfg->nx + 31) >> TILE_X_SHIFT;
  L.nty = (cfg->ny + 3) >> TILE_Y_SHIFT;
  L.ntz = (cfg->nz + 3) >> TILE_Z_SHIFT;
  const size_t sp = cfg->storage == STORE_F32 ? 4 : 2;
  L.pop = dalloc(h, h->lattice_mem, (size_t)Q * N * sp);
  L.uw = (float4*)dalloc(h, h->lattice_mem, sizeof(float4) * N);
  h->gbuf = (float4*)dalloc(h, h->lattice_mem, sizeof(float4) * N);
  h->fbuf = (uint8_t*)dalloc(h, h->lattice_mem, (size_t)tiles(L));
  L.g = h->gbuf;  // every view of the lattice (steps, stages, server) carries them
  L.flags = h->fbuf;
  L.status = (int*)dalloc(h, h->lattice_mem, 256);
  h->d_diag = (double*)dalloc(h, h->lattice_mem, 8 * sizeof(double));
  h->d_umax = (unsigned*)dalloc(h, h->lattice_mem, 256);
  if (!L.pop || !L.uw || !h->gbuf || !h->fbuf || !L.status || !h->d_diag ||
      !h->d_umax) {
    h->err = "device allocation failed";
    return bail(IBM_LBM_E_NOMEM);
  }
  {
    std::vector<RowInfo> rows = build_rows(L);
    h->n_rows = (int)rows.size();
    if (upload<RowInfo>(h, h->lattice_mem, &h->rows, rows.data(), rows.size())) return bail(IBM_LBM_E_NOMEM);
  }
  if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess)
    return bail(IBM_LBM_E_CUDA);
  if (transfer_configure() != cudaSuccess || couple_configure() != cudaSuccess) {
    cudaGetLastError();
    return bail(IBM_LBM_E_CUDA);
  }
  if (cudaMallocHost((void**)&h->h_diag, 8 * sizeof(double) + 2 * sizeof(unsigned) + sizeof(int)) != cudaSuccess)
    return bail(IBM_LBM_E_NOMEM);
  h->h_umax = reinterpret_cast<unsigned*>(h->h_diag + 8);
  h->h_status = reinterpret_cast<int*>(h->h_umax + 2);
  if (cudaMemsetAsync(L.status, 0, sizeof(int), h->stream) != cudaSuccess) return bail(IBM_LBM_E_CUDA);
  int rc = ibm_lbm_set_lattice(h, nullptr, nullptr);
  if (rc) return bail(rc);
  *out = h;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_destroy(ibm_lbm_t* h) {
  if (!h) return IBM_LBM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto e : h->events) cudaEventDestroy(e);
  h->events.clear();
  drop_graphs(h);
  release_pool(h, h->morse_mem);
  release_pool(h, h->marker_mem);
  release_pool(h, h->lattice_mem);
  if (h->h_diag) cudaFreeHost(h->h_diag);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_lattice(ibm_lbm_t* h, const double* rho, const double* u) {
  if (!h) return IBM_LBM_E_ARG;
  LatticeDev& L = h->L;
  const size_t N = (size_t)L.N;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  // the caller's FP64 arrays go to the device as they are and are converted
  // there (a host conversion loop over N cells costs more than the copy)
  std::vector<Alloc> tmp;
  double* d_rho = rho ? (double*)dalloc(h, tmp, sizeof(double) * N) : nullptr;
  double* d_u = u ? (double*)dalloc(h, tmp, sizeof(double) * 3 * N) : nullptr;
  if ((rho && !d_rho) || (u && !d_u)) {
    release_pool(h, tmp);
    return fail(h, IBM_LBM_E_NOMEM, "set_lattice: device allocation failed");
  }
  touch_pages(rho, sizeof(double) * N, false);
  touch_pages(u, sizeof(double) * 3 * N, false);
  int rc = IBM_LBM_OK;
  if (rho && cudaMemcpyAsync(d_rho, rho, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (!rc && u && cudaMemcpyAsync(d_u, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (!rc) {
    launch_set_moments(L, d_rho, d_u, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IBM_LBM_E_CUDA;
  }
  release_pool(h, tmp);
  if (rc) return fail(h, rc, "set_lattice: CUDA error");
  launch_init_equilibrium(L, h->cfg.storage, h->stream);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemsetAsync(h->gbuf, 0, sizeof(float4) * N, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->fbuf, 0, (size_t)tiles(L), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(L.status, 0, sizeof(int), h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->steps = 0;
  h->odd_next = false;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_populations(ibm_lbm_t* h, const double* f) {
  if (!h || !f) return fail(h, IBM_LBM_E_ARG, "null argument");
  std::vector<Alloc> tmp;
  const size_t bytes = sizeof(double) * Q * (size_t)h->L.N;
  double* d = (double*)dalloc(h, tmp, bytes);
  if (!d) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
  int rc = IBM_LBM_OK;
  if (cudaMemcpyAsync(d, f, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) rc = IBM_LBM_E_CUDA;
  if (!rc) {
    launch_import(h->L, h->cfg.storage, d, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IBM_LBM_E_CUDA;
  }
  release_pool(h, tmp);
  if (rc) return fail(h, rc, "set_populations: CUDA error");
  // the parity restarts: clear the force density and its flags
  CUDA_TRY(h, cudaMemsetAsync(h->gbuf, 0, sizeof(float4) * (size_t)h->L.N, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->fbuf, 0, (size_t)tiles(h->L), h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->odd_next = false;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_populations(ibm_lbm_t* h, double* f) {
  if (!h || !f) return fail(h, IBM_LBM_E_ARG, "null argument");
  std::vector<Alloc> tmp;
  const size_t bytes = sizeof(double) * Q * (size_t)h->L.N;
  double* d = (double*)dalloc(h, tmp, bytes);
  if (!d) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
  launch_export(h->L, h->cfg.storage, h->odd_next, d, h->stream);
  int rc = IBM_LBM_OK;
  if (cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  release_pool(h, tmp);
  if (rc) return fail(h, rc, "get_populations: CUDA error");
  return IBM_LBM_OK;
}

// Forget the markers, bodies, template and Morse lists (and the graphs that
// captured them): the handle is then a lattice without markers.
static void clear_markers(ibm_lbm_t* h) {
  drop_graphs(h);
  release_pool(h, h->morse_mem);
  release_pool(h, h->marker_mem);
  h->m = MarkersDev{};
  h->morse_ready = false;
  h->owner = nullptr;
  h->solid_v = nullptr;
  h->filament_list = nullptr;
  h->n_filaments = 0;
  h->n_bodies = 0;
  h->d_bodies = nullptr;
  h->h_bodies.clear();
  h->mesh = MeshDev{};
  h->membrane_list = h->rigid_list = nullptr;
  h->n_membranes = h->n_rigids = 0;
  h->groups = nullptr;
  h->n_groups = 0;
  h->boxes = nullptr;
  h->couple_items = nullptr;
  h->n_couple = 0;
  h->couple_order = nullptr;
  h->need_zero_F = false;
}

// set_markers after the old markers are gone; on error the caller clears
// whatever this allocated, so that a failed call leaves no half-built state.
static int set_markers_into(ibm_lbm_t* h, const ibm_lbm_mesh* mesh, int32_t n_bodies, const ibm_lbm_body* bodies,
                     int64_t n_markers, const double* X) {
  const int M = (int)n_markers;
  // validate bodies
  std::vector<std::pair<int64_t, int64_t>> ranges;
  bool any_membrane = false, any_rigid = false;
  int64_t covered = 0;
  for (int b = 0; b < n_bodies; ++b) {
    const ibm_lbm_body& B = bodies[b];
    if (B.first < 0 || B.count <= 0 || B.first + B.count > n_markers)
      return fail(h, IBM_LBM_E_ARG, "set_markers: body marker range out of bounds");
    if (B.kind == IBM_LBM_BODY_MEMBRANE) {
      any_membrane = true;
      if (!mesh) return fail(h, IBM_LBM_E_ARG, "set_markers: membrane body without a mesh");
      if (B.count != mesh->n_vertices)
        return fail(h, IBM_LBM_E_ARG, "set_markers: membrane marker count != mesh vertex count");
    } else if (B.kind == IBM_LBM_BODY_RIGID || B.kind == IBM_LBM_BODY_RIGID_DIRECT) {
      any_rigid = true;
      if (!(B.mass > 0) || !(B.inertia[0] > 0) || !(B.inertia[1] > 0) || !(B.inertia[2] > 0) || !(B.kappa >= 0))
        return fail(h, IBM_LBM_E_ARG, "set_markers: rigid body needs mass, inertia > 0 and kappa >= 0");
    } else if (B.kind == IBM_LBM_BODY_FILAMENT) {
      if (B.count < 2 || !(B.l0 > 0) || !(B.kBT_p >= 0) || !(B.k_b >= 0))
        return fail(h, IBM_LBM_E_ARG, "set_markers: filament needs >= 2 beads, l0 > 0, kBT_p >= 0 and k_b >= 0");
    } else {
      return fail(h, IBM_LBM_E_ARG, "set_markers: unknown body kind");
    }
    ranges.push_back({B.first, B.first + B.count});
    covered += B.count;
  }
  std::sort(ranges.begin(), ranges.end());
  for (size_t i = 1; i < ranges.size(); ++i)
    if (ranges[i].first < ranges[i - 1].second) return fail(h, IBM_LBM_E_ARG, "set_markers: bodies overlap");
  HostMesh hm;
  if (any_membrane) {
    std::string why;
    if (!build_mesh(mesh, hm, why)) return fail(h, IBM_LBM_E_ARG, why);
    if (hm.edges.size() >= 16384 || (size_t)mesh->n_triangles >= 16384)
      return fail(h, IBM_LBM_E_ARG, "set_markers: membrane template has too many edges or triangles");
  }
  // floor(X) of every coordinate must fit the stencil cache's int32
  for (size_t i = 0; i < 3 * (size_t)M; ++i)
    if (!(std::fabs(X[i]) < 1073741824.0))
      return fail(h, IBM_LBM_E_ARG, "set_markers: positions must be finite with |X| < 2^30");
  int rc;
  // marker arrays
  h->m.M = M;
  if ((rc = upload<double>(h, h->marker_mem, &h->m.X, X, 3 * (size_t)M))) return rc;
  h->m.U = (float4*)dalloc(h, h->marker_mem, sizeof(float4) * (size_t)M);
  h->m.F = (float4*)dalloc(h, h->marker_mem, sizeof(float4) * (size_t)M);
  h->m.cell = (int*)dalloc(h, h->marker_mem, sizeof(int) * 3 * (size_t)M);
  h->m.frac = (float*)dalloc(h, h->marker_mem, sizeof(float) * 3 * (size_t)M);
  if (!h->m.U || !h->m.F || !h->m.cell || !h->m.frac) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
  launch_stencil_cache(h->m, h->stream);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemset(h->m.U, 0, sizeof(float4) * (size_t)std::max(M, 1)));
  CUDA_TRY(h, cudaMemset(h->m.F, 0, sizeof(float4) * (size_t)std::max(M, 1)));
  // rigid body-frame offsets r_k = R^T (X_k - C)
  if (any_rigid) {
    std::vector<double> ref(3 * (size_t)M, 0.0);
    for (int b = 0; b < n_bodies; ++b) {
      const ibm_lbm_body& B = bodies[b];
      if (B.kind != IBM_LBM_BODY_RIGID && B.kind != IBM_LBM_BODY_RIGID_DIRECT) continue;
      double R[3][3];
      quat_matrix(B.quat, R);
      for (int64_t k = B.first; k < B.first + B.count; ++k) {
        const double d[3] = {X[k] - B.center[0], X[M + k] - B.center[1], X[2 * (size_t)M + k] - B.center[2]};
        for (int a = 0; a < 3; ++a) ref[a * (size_t)M + k] = R[0][a] * d[0] + R[1][a] * d[1] + R[2][a] * d[2];
      }
    }
    double* dref = nullptr;
    if ((rc = upload<double>(h, h->marker_mem, &dref, ref.data(), ref.size()))) return rc;
    h->m.ref = dref;
  }
  // body table
  std::vector<BodyDev> bd(std::max(n_bodies, 1));
  for (int b = 0; b < n_bodies; ++b) {
    const ibm_lbm_body& B = bodies[b];
    BodyDev& D = bd[b];
    D.kind = B.kind;
    D.first = (int)B.first;
    D.count = (int)B.count;
    D.kBT_p = (float)B.kBT_p; D.k_b = (float)B.k_b; D.k_l = (float)B.k_l; D.k_g = (float)B.k_g; D.k_v = (float)B.k_v;
    D.kappa = B.kappa; D.mass = B.mass;
    D.l0 = (float)B.l0;
    for (int a = 0; a < 3; ++a) {
      D.inertia[a] = B.inertia[a]; D.center[a] = B.center[a]; D.vel[a] = B.vel[a]; D.omega[a] = B.omega[a];
    }
    for (int a = 0; a < 4; ++a) D.quat[a] = B.quat[a];
    h->h_bodies.push_back(B);
  }
  if ((rc = upload<BodyDev>(h, h->marker_mem, &h->d_bodies, bd.data(), bd.size()))) return rc;
  h->n_bodies = n_bodies;
  {
    std::vector<int> mem, rig, fil;
    std::vector<int> own((size_t)std::max(M, 1), -1);
    for (int b = 0; b < n_bodies; ++b) {
      const int kind = bodies[b].kind;
      const bool rigid = kind == IBM_LBM_BODY_RIGID || kind == IBM_LBM_BODY_RIGID_DIRECT;
      (kind == IBM_LBM_BODY_MEMBRANE ? mem : rigid ? rig : fil).push_back(b);
      if (!rigid)
        for (int64_t k = bodies[b].first; k < bodies[b].first + bodies[b].count; ++k) own[k] = b;
    }
    h->n_membranes = (int)mem.size();
    h->n_rigids = (int)rig.size();
    h->n_filaments = (int)fil.size();
    if ((rc = upload<int>(h, h->marker_mem, &h->membrane_list, mem.data(), mem.size()))) return rc;
    if ((rc = upload<int>(h, h->marker_mem, &h->rigid_list, rig.data(), rig.size()))) return rc;
    if ((rc = upload<int>(h, h->marker_mem, &h->filament_list, fil.data(), fil.size()))) return rc;
    if ((rc = upload<int>(h, h->marker_mem, &h->owner, own.data(), own.size()))) return rc;
  }
  // mesh
  if (any_membrane) {
    // pack the topology into 16-byte-aligned sections of one buffer
    std::vector<unsigned char> buf;
    auto section = [&](const void* src, size_t bytes) {
      const int off = (int)buf.size();
      buf.resize(buf.size() + ((bytes + 15) / 16) * 16, 0);
      if (bytes) std::memcpy(buf.data() + off, src, bytes);
      return off;
    };
    std::vector<ushort4> e16(hm.edges.size());
    std::vector<ushort2> et16(hm.edges.size());
    for (size_t e = 0; e < hm.edges.size(); ++e) {
      e16[e] = make_ushort4(hm.edges[e].x, hm.edges[e].y, hm.edges[e].z, hm.edges[e].w);
      et16[e] = make_ushort2(hm.edge_tris[e].x, hm.edge_tris[e].y);
    }
    std::vector<ushort4> t16(hm.tris.size());
    for (size_t t = 0; t < hm.tris.size(); ++t) t16[t] = make_ushort4(hm.tris[t].x, hm.tris[t].y, hm.tris[t].z, 0);
    auto to16 = [](const std::vector<int>& v) { return std::vector<unsigned short>(v.begin(), v.end()); };
    const auto ves = to16(hm.v_edge_start), vel = to16(hm.v_edge), vts = to16(hm.v_tri_start), vtl = to16(hm.v_tri);
    MeshDev& D = h->mesh;
    D.off_edges = section(e16.data(), e16.size() * sizeof(ushort4));
    D.off_edge_tris = section(et16.data(), et16.size() * sizeof(ushort2));
    D.off_edge_rest = section(hm.edge_rest.data(), hm.edge_rest.size() * sizeof(float4));
    D.off_tris = section(t16.data(), t16.size() * sizeof(ushort4));
    D.off_area0 = section(hm.area0.data(), hm.area0.size() * sizeof(float));
    D.off_ve_start = section(ves.data(), ves.size() * 2);
    D.off_ve = section(vel.data(), vel.size() * 2);
    D.off_vt_start = section(vts.data(), vts.size() * 2);
    D.off_vt = section(vtl.data(), vtl.size() * 2);
    D.packed_bytes = (int)buf.size();
    unsigned char* dpk = nullptr;
    if ((rc = upload<unsigned char>(h, h->marker_mem, &dpk, buf.data(), buf.size()))) return rc;
    D.packed = dpk;
    D.nv = mesh->n_vertices;
    D.nt = mesh->n_triangles;
    D.ne = (int)hm.edges.size();
    D.work_floats = (int)membrane_work_floats(D.nv, D.nt, D.ne);
    D.A0 = (float)hm.A0;
    D.V0 = (float)hm.V0;
    int most = 1;  // contributions a vertex receives: its edge roles and triangles
    for (int v = 0; v < D.nv; ++v)
      most = std::max(most, hm.v_edge_start[v + 1] - hm.v_edge_start[v] + hm.v_tri_start[v + 1] - hm.v_tri_start[v]);
    D.qcap = (float)((2147483647.0 - 4096.0) / (double)most);
    int dev = 0, optin = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (forces_configure(D, (size_t)optin) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, IBM_LBM_E_ARG, "set_markers: membrane template too large for one thread block's shared memory");
    }
  }
  // transfer groups: bodies in chunks of BODY_GROUP, tracer runs in chunks of TRACER_GROUP
  {
    std::vector<MarkerGroup> groups;
    std::vector<std::pair<int64_t, int>> cuts;  // (first marker, body) in marker order
    for (int b = 0; b < n_bodies; ++b) cuts.push_back({bodies[b].first, b});
    std::sort(cuts.begin(), cuts.end());
    int64_t pos = 0;
    auto add_run = [&](int64_t a, int64_t b, int step, int flags) {
      for (int64_t s0 = a; s0 < b; s0 += step)
        groups.push_back({(int)s0, (int)std::min<int64_t>(step, b - s0), flags});
    };
    for (auto& c : cuts) {
      const ibm_lbm_body& B = bodies[c.second];
      add_run(pos, B.first, TRACER_GROUP, 0);
      add_run(B.first, B.first + B.count, BODY_GROUP, B.kind == IBM_LBM_BODY_RIGID_DIRECT ? GROUP_FIXED : 0);
      pos = B.first + B.count;
    }
    add_run(pos, n_markers, TRACER_GROUP, 0);
    // Transfer blocks in the order of a Morton curve through the groups'
    // mean positions (cells / 8 per axis, periodic x wrapped): blocks that
    // run close in time then work on neighbouring cells, so the overlapping
    // parts of their boxes are served from L2 rather than HBM.
    {
      const double nxd = (double)h->cfg.nx;
      auto spread_bits = [](uint32_t v) {  // 10 bits -> every third of 30
        uint64_t x = v & 0x3ffu;
        x = (x | (x << 16)) & 0x30000ffull;
        x = (x | (x << 8)) & 0x300f00full;
        x = (x | (x << 4)) & 0x30c30c3ull;
        x = (x | (x << 2)) & 0x9249249ull;
        return x;
      };
      std::vector<std::pair<uint64_t, size_t>> key(groups.size());
      for (size_t g = 0; g < groups.size(); ++g) {
        double c[3] = {0.0, 0.0, 0.0};
        for (int k = groups[g].first; k < groups[g].first + groups[g].count; ++k)
          for (int a = 0; a < 3; ++a) c[a] += X[a * (size_t)M + k];
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
          double v = c[a] / (double)groups[g].count;
          if (a == 0) v -= nxd * std::floor(v / nxd);
          q[a] = (uint32_t)std::min(1023.0, std::max(0.0, v / 8.0));
        }
        key[g] = {spread_bits(q[0]) | (spread_bits(q[1]) << 1) | (spread_bits(q[2]) << 2), g};
      }
      std::stable_sort(key.begin(), key.end(),
                       [](const std::pair<uint64_t, size_t>& a, const std::pair<uint64_t, size_t>& b) {
                         return a.first < b.first;
                       });
      std::vector<MarkerGroup> ordered(groups.size());
      for (size_t g = 0; g < groups.size(); ++g) ordered[g] = groups[key[g].second];
      groups.swap(ordered);
    }
    h->n_groups = (int)groups.size();
    if ((rc = upload<MarkerGroup>(h, h->marker_mem, &h->groups, groups.data(), groups.size()))) return rc;
    // fused path: every marker belongs to a membrane whose template fits the
    // fused kernel, one transfer group per body
    bool fused = n_bodies > 0 && covered == n_markers && any_membrane && couple_fits(h->mesh);
    for (int b = 0; b < n_bodies && fused; ++b) fused = bodies[b].kind == IBM_LBM_BODY_MEMBRANE;
    if (fused) {
      std::unordered_map<int, int> body_of_first;
      for (int b = 0; b < n_bodies; ++b) body_of_first[(int)bodies[b].first] = b;
      // items[g] = (body, g) for every group g in order: the fused kernel's
      // block g reads group g and its box directly
      std::vector<int2> items;
      for (size_t g = 0; g < groups.size() && fused; ++g) {
        auto it = body_of_first.find(groups[g].first);
        if (it == body_of_first.end() || groups[g].count != (int)bodies[it->second].count) fused = false;
        else items.push_back(make_int2(it->second, (int)g));
      }
      if (fused && (int)items.size() == n_bodies && items.size() == groups.size()) {
        if ((rc = upload<int2>(h, h->marker_mem, &h->couple_items, items.data(), items.size()))) return rc;
        h->couple_order = (unsigned char*)dalloc(h, h->marker_mem, couple_order_bytes(h->mesh) * items.size());
        if (!h->couple_order) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
        h->n_couple = (int)items.size();
      }
    }
    h->boxes = (int4*)dalloc(h, h->marker_mem, sizeof(int4) * 2 * std::max<size_t>(1, groups.size()));
    if (!h->boxes) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
    // no box until the first spreading: an interpolation run before it (the
    // stage interface allows that) takes the per-marker path
    CUDA_TRY(h, cudaMemset(h->boxes, 0, sizeof(int4) * 2 * std::max<size_t>(1, groups.size())));
  }
  h->need_zero_F = covered < n_markers;
  if (h->morse_rc > 0.0) return prepare_morse(h);
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_markers(ibm_lbm_t* h, const ibm_lbm_mesh* mesh, int32_t n_bodies, const ibm_lbm_body* bodies,
                                    int64_t n_markers, const double* X) {
  if (!h) return IBM_LBM_E_ARG;
  if (n_bodies < 0 || n_markers < 0 || n_markers >= (1LL << 31) || (n_markers > 0 && !X) ||
      (n_bodies > 0 && !bodies))
    return fail(h, IBM_LBM_E_ARG, "set_markers: bad counts or null arrays");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  clear_markers(h);
  const int rc = set_markers_into(h, mesh, n_bodies, bodies, n_markers, X);
  if (rc != IBM_LBM_OK) {
    const std::string why = h->err;
    clear_markers(h);
    h->err = why;
  }
  return rc;
}

static int impl_ibm_lbm_solid_steps(ibm_lbm_t* h, int64_t n_steps, double dt, double gamma, double mass, const double* f_ext) {
  if (!h) return IBM_LBM_E_ARG;
  if (n_steps < 0 || !(dt > 0.0) || !(gamma >= 0.0) || !(mass > 0.0))
    return fail(h, IBM_LBM_E_ARG, "solid_steps: needs n_steps >= 0, dt > 0, gamma >= 0, mass > 0");
  if (h->n_rigids > 0) return fail(h, IBM_LBM_E_STATE, "solid_steps: rigid bodies need the fluid");
  const size_t M = (size_t)h->m.M;
  if (M == 0 || n_steps == 0) return IBM_LBM_OK;
  cudaStream_t st = h->stream;
  CUDA_TRY(h, cudaStreamSynchronize(st));
  if (!h->solid_v) {
    h->solid_v = (double*)dalloc(h, h->marker_mem, sizeof(double) * 3 * M);
    if (!h->solid_v) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
    CUDA_TRY(h, cudaMemset(h->solid_v, 0, sizeof(double) * 3 * M));
  }
  std::vector<Alloc> tmp;
  double* fe = nullptr;
  if (f_ext) {
    fe = (double*)dalloc(h, tmp, sizeof(double) * 3 * M);
    if (!fe) return fail(h, IBM_LBM_E_NOMEM, "device allocation failed");
    if (cudaMemcpy(fe, f_ext, sizeof(double) * 3 * M, cudaMemcpyHostToDevice) != cudaSuccess) {
      release_pool(h, tmp);
      return fail(h, IBM_LBM_E_CUDA, "solid_steps: copy of f_ext failed");
    }
  }
  for (int64_t s = 0; s < n_steps; ++s) {
    enqueue_forces(h, st);
    launch_solid_half(h->m, h->solid_v, fe, dt, gamma, mass, true, st);
    enqueue_forces(h, st);
    launch_solid_half(h->m, h->solid_v, fe, dt, gamma, mass, false, st);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release_pool(h, tmp);
  if (e != cudaSuccess) return fail(h, IBM_LBM_E_CUDA, std::string("solid_steps: ") + cudaGetErrorString(e));
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_morse(ibm_lbm_t* h, double D0, double alpha, double r0, double rc) {
  if (!h) return IBM_LBM_E_ARG;
  if (rc > 0.0 && (!(D0 >= 0.0) || !(alpha > 0.0) || !std::isfinite(r0) || !std::isfinite(rc)))
    return fail(h, IBM_LBM_E_ARG, "set_morse: needs D0 >= 0, alpha > 0 and finite r0, rc");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  h->morse_D0 = D0;
  h->morse_alpha = alpha;
  h->morse_r0 = r0;
  h->morse_rc = rc > 0.0 ? rc : 0.0;
  release_pool(h, h->morse_mem);
  h->morse_ready = false;
  if (h->morse_rc > 0.0 && h->owner) return prepare_morse(h);
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_step_async(ibm_lbm_t* h, int64_t n_steps) {
  if (!h) return IBM_LBM_E_ARG;
  return enqueue_steps(h, n_steps);
}

static int impl_ibm_lbm_synchronize(ibm_lbm_t* h) {
  if (!h) return IBM_LBM_E_ARG;
  return finish_diagnostics(h);
}

static int impl_ibm_lbm_step(ibm_lbm_t* h, int64_t n_steps) {
  if (!h) return IBM_LBM_E_ARG;
  int rc = enqueue_steps(h, n_steps);
  if (rc) return rc;
  return finish_diagnostics(h);
}

static int impl_ibm_lbm_run_stage(ibm_lbm_t* h, int32_t stage) {
  if (!h) return IBM_LBM_E_ARG;
  cudaStream_t st = h->stream;
  // The interpolation gathers from the stencil boxes the last spreading
  // computed; they hold the markers only while no stage has moved them since
  // (the interpolation advects, the direct rigid forcing places markers).
  // Otherwise the boxes are cleared first and every marker takes the
  // per-marker path.
  switch (stage) {
    case IBM_LBM_STAGE_FORCES:
      enqueue_forces(h, st);
      h->boxes_valid = false;
      break;
    case IBM_LBM_STAGE_SPREAD: {
      const LatticeDev L = lat(h, h->odd_next);
      CUDA_TRY(h, cudaMemsetAsync(L.flags, 0, (size_t)tiles(L), st));
      launch_spread(L, h->m, h->groups, h->n_groups, h->boxes, st);
      h->boxes_valid = true;
      break;
    }
    case IBM_LBM_STAGE_COLLIDE:
      launch_collide(lat(h, h->odd_next), h->rows, h->n_rows, h->cfg.storage, h->odd_next, true, st);
      h->odd_next = !h->odd_next;
      break;
    case IBM_LBM_STAGE_INTERP:
      if (!h->boxes_valid && h->n_groups > 0)
        CUDA_TRY(h, cudaMemsetAsync(h->boxes, 0, sizeof(int4) * 2 * (size_t)h->n_groups, st));
      launch_interpolate(h->L, h->m, h->groups, h->n_groups, h->boxes, st);
      h->boxes_valid = false;
      h->steps += 1;
      break;
    default:
      return fail(h, IBM_LBM_E_ARG, "unknown stage");
  }
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaStreamSynchronize(st));
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_marker_forces(ibm_lbm_t* h, const double* F) {
  if (!h || (!F && h->m.M > 0)) return fail(h, IBM_LBM_E_ARG, "null argument");
  const size_t M = (size_t)h->m.M;
  std::vector<float4> tmp(M);
  for (size_t k = 0; k < M; ++k) tmp[k] = make_float4((float)F[k], (float)F[M + k], (float)F[2 * M + k], 0.f);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (M) CUDA_TRY(h, cudaMemcpy(h->m.F, tmp.data(), sizeof(float4) * M, cudaMemcpyHostToDevice));
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_force_density(ibm_lbm_t* h, double* g) {
  if (!h || !g) return fail(h, IBM_LBM_E_ARG, "null argument");
  const size_t N = (size_t)h->L.N;
  std::vector<float4> tmp(N);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(tmp.data(), h->gbuf, sizeof(float4) * N, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < N; ++i) {
    g[i] = tmp[i].x; g[N + i] = tmp[i].y; g[2 * N + i] = tmp[i].z;
  }
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_fields(ibm_lbm_t* h, double* rho, double* u) {
  if (!h) return IBM_LBM_E_ARG;
  const LatticeDev& L = h->L;
  const size_t N = (size_t)L.N;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (!rho && !u) return IBM_LBM_OK;
  // expanded to the FP64 layout on the device, then one copy per array
  std::vector<Alloc> tmp;
  double* d_rho = rho ? (double*)dalloc(h, tmp, sizeof(double) * N) : nullptr;
  double* d_u = u ? (double*)dalloc(h, tmp, sizeof(double) * 3 * N) : nullptr;
  if ((rho && !d_rho) || (u && !d_u)) {
    release_pool(h, tmp);
    return fail(h, IBM_LBM_E_NOMEM, "get_fields: device allocation failed");
  }
  launch_get_moments(L, d_rho, d_u, h->stream);
  // while the kernel runs: take the page faults of freshly allocated output
  // arrays on several threads (the copy would take them one by one)
  touch_pages(rho, sizeof(double) * N, true);
  touch_pages(u, sizeof(double) * 3 * N, true);
  int rc = IBM_LBM_OK;
  if (rho && cudaMemcpyAsync(rho, d_rho, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (!rc && u && cudaMemcpyAsync(u, d_u, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IBM_LBM_E_CUDA;
  release_pool(h, tmp);
  if (rc) return fail(h, rc, "get_fields: CUDA error");
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_markers(ibm_lbm_t* h, double* X, double* U, double* F) {
  if (!h) return IBM_LBM_E_ARG;
  const size_t M = (size_t)h->m.M;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (M == 0) return IBM_LBM_OK;
  // U and F expanded to the FP64 [3][M] layout on the device
  std::vector<Alloc> tmp;
  double* dU = U ? (double*)dalloc(h, tmp, sizeof(double) * 3 * M) : nullptr;
  double* dF = F ? (double*)dalloc(h, tmp, sizeof(double) * 3 * M) : nullptr;
  if ((U && !dU) || (F && !dF)) {
    release_pool(h, tmp);
    return fail(h, IBM_LBM_E_NOMEM, "get_markers: device allocation failed");
  }
  if (U) launch_expand_xyz(h->m.U, dU, (int)M, h->stream);
  if (F) launch_expand_xyz(h->m.F, dF, (int)M, h->stream);
  touch_pages(X, sizeof(double) * 3 * M, true);
  touch_pages(U, sizeof(double) * 3 * M, true);
  touch_pages(F, sizeof(double) * 3 * M, true);
  int rc = IBM_LBM_OK;
  if (X && cudaMemcpyAsync(X, h->m.X, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (!rc && U && cudaMemcpyAsync(U, dU, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (!rc && F && cudaMemcpyAsync(F, dF, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = IBM_LBM_E_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IBM_LBM_E_CUDA;
  release_pool(h, tmp);
  if (rc) return fail(h, rc, "get_markers: CUDA error");
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_bodies(ibm_lbm_t* h, ibm_lbm_body* bodies, int32_t n_bodies) {
  if (!h || n_bodies != h->n_bodies || (n_bodies > 0 && !bodies))
    return fail(h, IBM_LBM_E_ARG, "get_bodies: count mismatch");
  if (n_bodies == 0) return IBM_LBM_OK;
  std::vector<BodyDev> bd(n_bodies);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(bd.data(), h->d_bodies, sizeof(BodyDev) * n_bodies, cudaMemcpyDeviceToHost));
  for (int b = 0; b < n_bodies; ++b) {
    ibm_lbm_body B = h->h_bodies[b];
    for (int a = 0; a < 3; ++a) {
      B.center[a] = bd[b].center[a]; B.vel[a] = bd[b].vel[a]; B.omega[a] = bd[b].omega[a];
    }
    for (int a = 0; a < 4; ++a) B.quat[a] = bd[b].quat[a];
    bodies[b] = B;
  }
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_timing(ibm_lbm_t* h, int64_t max_steps) {
  if (!h || max_steps < 0 || max_steps > (1 << 22)) return fail(h, IBM_LBM_E_ARG, "set_timing: bad step count");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (auto e : h->events) cudaEventDestroy(e);
  h->events.clear();
  h->timed_steps = 0;
  h->timed_odd.clear();
  h->timed_fused.clear();
  h->timing = max_steps > 0;
  for (int64_t i = 0; i < 5 * max_steps; ++i) {
    cudaEvent_t e;
    CUDA_TRY(h, cudaEventCreate(&e));
    h->events.push_back(e);
  }
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_set_timing_fused(ibm_lbm_t* h, int on) {
  if (!h) return IBM_LBM_E_ARG;
  h->timing_fused = on != 0;
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_timing(ibm_lbm_t* h, double out[6]) {
  if (!h || !out) return IBM_LBM_E_ARG;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < 6; ++k) out[k] = 0.0;
  for (size_t s = 0; s < h->timed_steps; ++s)
    for (int k = h->timed_fused[s] ? 2 : 0; k < 4; ++k) {
      float ms = 0.f;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, h->events[5 * s + k], h->events[5 * s + k + 1]));
      out[k] += ms;
      if (k == 2 && h->timed_odd[s]) out[5] += ms;
    }
  out[4] = (double)h->timed_steps;
  h->timed_steps = 0;
  h->timed_odd.clear();
  h->timed_fused.clear();
  return IBM_LBM_OK;
}

static int impl_ibm_lbm_get_diagnostics(ibm_lbm_t* h, double out[8]) {
  if (!h || !out) return IBM_LBM_E_ARG;
  int rc = enqueue_diagnostics(h);
  if (rc) return rc;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->diag_pending = false;
  float umax2;
  std::memcpy(&umax2, h->h_umax, sizeof(float));
  out[0] = h->h_diag[4] + h->h_diag[0];
  out[1] = h->h_diag[1];
  out[2] = h->h_diag[2];
  out[3] = h->h_diag[3];
  out[4] = std::sqrt((double)umax2);
  out[5] = (double)h->steps;
  out[6] = h->h_diag[4];
  out[7] = 0.0;
  return IBM_LBM_OK;
}


int ibm_lbm_create(const ibm_lbm_config* cfg, const ibm_lbm_allocator* alloc, void* stream, ibm_lbm_t** out) {
  return abi_guard(nullptr, [&]() -> int { return impl_ibm_lbm_create(cfg, alloc, stream, out); });
}

int ibm_lbm_destroy(ibm_lbm_t* h) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_destroy(h); });
}

int ibm_lbm_set_lattice(ibm_lbm_t* h, const double* rho, const double* u) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_lattice(h, rho, u); });
}

int ibm_lbm_set_populations(ibm_lbm_t* h, const double* f) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_populations(h, f); });
}

int ibm_lbm_get_populations(ibm_lbm_t* h, double* f) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_populations(h, f); });
}

int ibm_lbm_set_markers(ibm_lbm_t* h, const ibm_lbm_mesh* mesh, int32_t n_bodies, const ibm_lbm_body* bodies,
                        int64_t n_markers, const double* X) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_markers(h, mesh, n_bodies, bodies, n_markers, X); });
}

int ibm_lbm_solid_steps(ibm_lbm_t* h, int64_t n_steps, double dt, double gamma, double mass, const double* f_ext) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_solid_steps(h, n_steps, dt, gamma, mass, f_ext); });
}

int ibm_lbm_set_morse(ibm_lbm_t* h, double D0, double alpha, double r0, double rc) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_morse(h, D0, alpha, r0, rc); });
}

int ibm_lbm_step_async(ibm_lbm_t* h, int64_t n_steps) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_step_async(h, n_steps); });
}

int ibm_lbm_synchronize(ibm_lbm_t* h) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_synchronize(h); });
}

int ibm_lbm_step(ibm_lbm_t* h, int64_t n_steps) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_step(h, n_steps); });
}

int ibm_lbm_run_stage(ibm_lbm_t* h, int32_t stage) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_run_stage(h, stage); });
}

int ibm_lbm_set_marker_forces(ibm_lbm_t* h, const double* F) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_marker_forces(h, F); });
}

int ibm_lbm_get_force_density(ibm_lbm_t* h, double* g) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_force_density(h, g); });
}

int ibm_lbm_get_fields(ibm_lbm_t* h, double* rho, double* u) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_fields(h, rho, u); });
}

int ibm_lbm_get_markers(ibm_lbm_t* h, double* X, double* U, double* F) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_markers(h, X, U, F); });
}

int ibm_lbm_get_bodies(ibm_lbm_t* h, ibm_lbm_body* bodies, int32_t n_bodies) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_bodies(h, bodies, n_bodies); });
}

int ibm_lbm_set_timing(ibm_lbm_t* h, int64_t max_steps) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_timing(h, max_steps); });
}

int ibm_lbm_set_timing_fused(ibm_lbm_t* h, int on) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_set_timing_fused(h, on); });
}

int ibm_lbm_get_timing(ibm_lbm_t* h, double out[6]) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_timing(h, out); });
}

int ibm_lbm_get_diagnostics(ibm_lbm_t* h, double out[8]) {
  return abi_guard(h, [&]() -> int { return impl_ibm_lbm_get_diagnostics(h, out); });
}
}  // extern "C"

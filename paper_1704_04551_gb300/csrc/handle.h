// Internal definition of the ibm_lbm handle, shared by the single-lattice C
// ABI (api.cu) and the batched server (serve.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ibm_lbm.h"
#include "common.cuh"
#include "morse.cuh"

namespace ibm {
constexpr int CHUNK = 16;          // steps per captured chunk graph (even)
constexpr int FUSED_LONG = 64;     // steps per long fused chunk graph (even)
constexpr int MAX_MESH_VERTICES = 4096;
constexpr int BODY_GROUP = 1024;   // markers per transfer block within a body
constexpr int TRACER_GROUP = 256;  // markers per transfer block for passive tracers

struct Alloc {
  void* p;
  size_t bytes;
};
}  // namespace ibm

struct ibm_lbm {
  using LatticeDev = ibm::LatticeDev;
  using RowInfo = ibm::RowInfo;
  using Alloc = ibm::Alloc;
  using MarkersDev = ibm::MarkersDev;
  using BodyDev = ibm::BodyDev;
  using MeshDev = ibm::MeshDev;
  using MarkerGroup = ibm::MarkerGroup;
  ibm_lbm_config cfg{};
  ibm_lbm_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  LatticeDev L{};                 // the lattice view every kernel receives
  float4* gbuf = nullptr;         // force density
  uint8_t* fbuf = nullptr;        // touched-tile flags
  RowInfo* rows = nullptr;        // fluid rows of the lattice
  int n_rows = 0;
  std::vector<Alloc> lattice_mem, marker_mem;
  size_t bytes = 0;
  // markers
  MarkersDev m{};
  int n_bodies = 0;
  BodyDev* d_bodies = nullptr;
  std::vector<ibm_lbm_body> h_bodies;
  MeshDev mesh{};
  int* membrane_list = nullptr;   // body indices of membranes / rigid bodies / filaments
  int* rigid_list = nullptr;
  int* filament_list = nullptr;
  int n_membranes = 0, n_rigids = 0, n_filaments = 0;
  int* owner = nullptr;           // [M] body of each membrane / filament marker, -1 otherwise
  double* solid_v = nullptr;      // [3][M] marker velocities of the solid-only dynamics (lazily allocated)
  // Morse excluded volume (off while rc <= 0)
  double morse_D0 = 0.0, morse_alpha = 0.0, morse_r0 = 0.0, morse_rc = 0.0;
  ibm::MorseDev morse{};
  bool morse_ready = false;       // cell-list buffers match the markers
  std::vector<Alloc> morse_mem;
  int n_sm = 0;
  MarkerGroup* groups = nullptr;  // transfer blocks
  int n_groups = 0;
  int4* boxes = nullptr;          // per group: stencil box origin and size
  // Fused coupling (suspensions of membranes only): one block per body
  // interpolates, computes the forces and spreads; the collision of
  // alternate steps reads the two force-density buffers in turn.
  int2* couple_items = nullptr;   // (body, its transfer group) in group order
  int n_couple = 0;               // > 0: the fused path applies to these markers
  // per fused body, left by its spreading for the next step's gather: the
  // vertices' residue counters and order (couple_order_bytes each)
  unsigned char* couple_order = nullptr;
  float4* gbuf2 = nullptr;        // second force density (allocated on first use)
  bool boxes_valid = false;       // boxes match the markers' current positions (stage interface)
  bool need_zero_F = false;
  // state
  long long steps = 0;
  bool odd_next = false;          // the array is in the post-even-step layout
  double* d_diag = nullptr;       // [8]
  unsigned* d_umax = nullptr;
  double* h_diag = nullptr;       // pinned [8]
  unsigned* h_umax = nullptr;     // pinned
  int* h_status = nullptr;        // pinned
  bool diag_pending = false;
  // per-stage timing (events between stages, direct launches)
  std::vector<cudaEvent_t> events;  // 5 per timed step
  std::vector<char> timed_odd;      // AA parity of each timed step
  std::vector<char> timed_fused;    // timed step on the fused path (no forces / spreading slots)
  size_t timed_steps = 0;
  bool timing = false;
  bool timing_fused = false;  // time the fused path where it applies
  // graphs
  cudaGraphExec_t g_chunk = nullptr;
  cudaGraphExec_t g_fused[2] = {nullptr, nullptr};  // fused chunks of FUSED_LONG and CHUNK steps
  cudaGraphExec_t g_single[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  std::string err;
};


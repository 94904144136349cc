/*
 * ibm_lbm.h — C ABI of the GB300 (sm_103a) coupled immersed-boundary /
 * lattice-Boltzmann time step of Tan, Sinno & Diamond, "A parallel fluid
 * solid coupling model using LAMMPS and Palabos based on the immersed
 * boundary method" (arXiv:1704.04551).
 *
 * One time step, in this order (the paper does not print the order; this
 * library and its test oracle use the same reading):
 *   1. marker forces at X^n — membrane forces -dU/dX of Eq. membrane-potential
 *      (Eqs. inPlanePotential, bendingEnergy, areaEnergy, volumeEnergy,
 *      Sec. 2.2), or a rigid body's penalty tether with a Newton-Euler update
 *      of the body (Sec. 2.3);
 *   2. spreading of marker forces to the lattice, Eq. ibmForceSpread, with the
 *      4-point cosine delta of Eq. deltaPhiSimple;
 *   3. D3Q19 BGK collision with Guo forcing and streaming, Eqs. lbm,
 *      BGKequilibrium, rho_u and the Guo term (Sec. 2.1), half-way
 *      bounce-back at walls;
 *   4. interpolation of the collision-time lattice velocity to the markers,
 *      Eq. ibmVelocityInterpret, and advection X^{n+1} = X^n + U.
 * These are the two coupling routines of the paper's List 1
 * (interpolateVelocity3D / spreadForce3D) plus the fluid and solid steps
 * they connect.
 *
 * Conventions (every entry point):
 *   - Lattice units: dx = dt = 1, fluid density ~1, c_s^2 = 1/3.
 *   - Cell index idx = x + nx*(y + ny*z); cell (x,y,z) sits at position
 *     (x,y,z). Scalar fields are [N], vector fields [3][N] (component
 *     major), populations [19][N], marker arrays [3][M]; all host arrays are
 *     dense, C order, owned by the caller, and only read or written during
 *     the call (the library keeps no host pointer).
 *   - D3Q19 order: 0 (0,0,0); 1,2 (+-1,0,0); 3,4 (0,+-1,0); 5,6 (0,0,+-1);
 *     7,8 +-(1,1,0); 9,10 +-(1,-1,0); 11,12 +-(1,0,1); 13,14 +-(1,0,-1);
 *     15,16 +-(0,1,1); 17,18 +-(0,1,-1). Weights 1/3, 1/18, 1/36.
 *   - Every call returns an ibm_lbm_status (0 = OK, negative = error) and
 *     never aborts; ibm_lbm_last_error() gives the message of the last
 *     failure on that handle. A handle may be used from one host thread at
 *     a time.
 *   - Device memory is owned by the handle and allocated at create /
 *     set_markers time through the caller's allocator (or cudaMalloc when
 *     none is given). Stepping allocates nothing.
 */
#ifndef IBM_LBM_H
#define IBM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IBM_LBM_OK = 0,
  IBM_LBM_E_ARG = -1,      /* invalid argument (sizes, ranges, mesh topology) */
  IBM_LBM_E_NOMEM = -2,    /* the allocator returned NULL */
  IBM_LBM_E_CUDA = -3,     /* a CUDA runtime call failed */
  IBM_LBM_E_UNSTABLE = -4, /* non-finite or |u| > 0.4 found by the end-of-call check */
  IBM_LBM_E_TIMEOUT = -5,  /* a bounded wait gave up */
  IBM_LBM_E_STATE = -6     /* call not valid in the handle's current state */
} ibm_lbm_status;

enum { IBM_LBM_STORE_F32 = 0, IBM_LBM_STORE_F16_DEV = 1, IBM_LBM_STORE_BF16_DEV = 2 };
enum { IBM_LBM_GEOM_PERIODIC = 0, IBM_LBM_GEOM_YWALLS = 1, IBM_LBM_GEOM_TUBE = 2 };
enum { IBM_LBM_BODY_MEMBRANE = 0, IBM_LBM_BODY_RIGID = 1, IBM_LBM_BODY_FILAMENT = 2, IBM_LBM_BODY_RIGID_DIRECT = 3 };
enum { IBM_LBM_STAGE_FORCES = 0, IBM_LBM_STAGE_SPREAD = 1, IBM_LBM_STAGE_COLLIDE = 2,
       IBM_LBM_STAGE_INTERP = 3 };

/* Device-memory provider. alloc returns a device pointer aligned to at
 * least 256 bytes, or NULL (the call that needed the memory then returns
 * IBM_LBM_E_NOMEM and releases what it took); release frees it. Called only
 * from the calls that take or return device memory (create, set_lattice,
 * set_populations, get_populations, set_markers, set_morse, solid_steps,
 * destroy, and the server's submit, advance and destroy), on the calling
 * thread. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*release)(void* ptr, void* ctx);
  void* ctx;
} ibm_lbm_allocator;

/* Lattice description (Sec. 2.1). */
typedef struct {
  int32_t nx, ny, nz;   /* cells; each >= 4, N = nx*ny*nz < 2^31 */
  int32_t geometry;     /* IBM_LBM_GEOM_*: periodic box; walls at y = -1/2 and
                           y = ny - 1/2 (periodic x, z); tube along x whose
                           solid cells lie farther than tube_radius from the
                           axis y = (ny-1)/2, z = (nz-1)/2 (periodic x) */
  double tau;           /* BGK relaxation time > 1/2; nu = (tau - 1/2)/3 (Eq. viscosity) */
  double wall_u[2];     /* x velocity of the y = -1/2 and y = ny - 1/2 walls */
  double tube_radius;
  double body_force[3]; /* uniform force density g0 added to the spread one */
  int32_t storage;      /* IBM_LBM_STORE_*: populations stored as FP32 deviations
                           f_i - w_i, or as FP16 / BF16 scaled deviations
                           K_i (f_i - w_i), K = 4, 16, 32 for rest, axis, diagonal;
                           all arithmetic is FP32 */
  int32_t device;       /* CUDA device ordinal */
} ibm_lbm_config;

/* One immersed body: a contiguous range of markers. Membranes use the
 * template mesh of ibm_lbm_set_markers (count == its vertex count). Rigid
 * bodies tether each marker to a body-fixed point (penalty reading of the
 * rigid coupling of Sec. 2.3, Eq. FSIRigid): force on the fluid
 * F_k = -kappa (X_k - X_k^ref), reaction on the body, explicit Newton-Euler
 * update of the pose. Direct-forcing rigid bodies use the paper's own FSI
 * force (Eq. FSIRigid): the force density on the solid at a marker is
 * rho_f (u(X) - U(X))/dt, u the fluid velocity interpolated there at the
 * last interpolation, U = V + omega x (X - C) the body's velocity; each
 * marker stands for a volume kappa (rho_f = dt = 1, so the nodal force on
 * the solid is kappa (u - U)), the fluid receives the opposite force, and
 * after the Newton-Euler update the markers are moved rigidly to the new
 * pose (they are not advected by the fluid). Filaments (polymer particles of Sec. 2.2) are bead
 * chains in marker order (count >= 2): each bond has the stretching energy
 * of Eq. inPlanePotential with l_m = 2 l0 and k_p = 1.25 (kBT/p) l0^2 (no
 * force at the rest length), each interior bead the bending energy
 * k_b (theta - pi)^2 of Eq. bendingEnergyWorm (theta the angle between its
 * two bonds; straight at rest). */
typedef struct {
  int32_t kind;                 /* IBM_LBM_BODY_* */
  int32_t pad;
  int64_t first, count;         /* marker range */
  double kBT_p, k_b, k_l, k_g, k_v;  /* membrane: kBT/p, bending, local/global
                                        area, volume moduli (Eqs. inPlanePotential,
                                        bendingEnergy, areaEnergy, volumeEnergy);
                                        filament: kBT/p and k_b */
  double kappa;                 /* rigid: tether stiffness; rigid direct: volume per marker */
  double mass, inertia[3];      /* rigid: mass and principal moments (body frame) */
  double center[3], quat[4];    /* rigid: centre, unit quaternion (w,x,y,z) body->world */
  double vel[3], omega[3];      /* rigid: velocity, angular velocity (world frame) */
  double l0;                    /* filament: rest bond length (> 0) */
} ibm_lbm_body;

/* Membrane template (Sec. 2.2): closed, consistently outward-oriented
 * triangle mesh. Rest edge lengths, rest dihedral angles, rest triangle
 * areas, rest total area and volume are taken from rest_X. */
typedef struct {
  int32_t n_vertices;      /* <= 4096, and 24 B per vertex + 16 B per triangle + 8 B per
                              edge must fit one thread block's shared memory (about
                              2800 vertices for a closed triangulation) */
  int32_t n_triangles;
  const int32_t* tris;     /* host [n_triangles][3], counter-clockwise seen from outside */
  const double* rest_X;    /* host [3][n_vertices] */
} ibm_lbm_mesh;

typedef struct ibm_lbm ibm_lbm_t;

/* Create a lattice at rest (rho = 1, u = 0 at equilibrium, Sec. 2.1).
 * alloc may be NULL (cudaMalloc/cudaFree). stream is a cudaStream_t or NULL
 * (the handle then creates its own non-blocking stream); all work of the
 * handle is ordered on that stream. Errors: E_ARG, E_NOMEM, E_CUDA. */
int ibm_lbm_create(const ibm_lbm_config* cfg, const ibm_lbm_allocator* alloc, void* stream,
                   ibm_lbm_t** out);

/* Synchronise the stream and release all device memory. NULL is a no-op. */
int ibm_lbm_destroy(ibm_lbm_t* h);

/* Initialise every fluid cell at equilibrium f = f^eq(rho, u) (Sec. 2.1,
 * Eq. BGKequilibrium). rho: host [N] or NULL (= 1); u: host [3][N] or NULL
 * (= 0). Resets the step counter and clears spread forces. */
int ibm_lbm_set_lattice(ibm_lbm_t* h, const double* rho, const double* u);

/* Raw populations f_i (not deviations), host [19][N] FP64, in the natural
 * (pre-collision) layout of the D3Q19 order above. set resets the step
 * parity; values are rounded to the storage format. */
int ibm_lbm_set_populations(ibm_lbm_t* h, const double* f);
int ibm_lbm_get_populations(ibm_lbm_t* h, double* f);

/* Markers, bodies and (optional) membrane template. mesh may be NULL when
 * no body is a membrane. X: host [3][n_markers], unwrapped coordinates in
 * lattice units, finite with |X| < 2^30. Markers outside every body are
 * passive tracers (zero force). Errors: E_ARG (overlapping or out-of-range
 * bodies, membrane count != n_vertices, non-manifold mesh, template too
 * large, a non-finite or too large position), E_NOMEM. The previous markers
 * are dropped first; after any error the handle holds no markers (a lattice
 * alone, which can still step) and none of the failed call's memory. */
int ibm_lbm_set_markers(ibm_lbm_t* h, const ibm_lbm_mesh* mesh, int32_t n_bodies,
                        const ibm_lbm_body* bodies, int64_t n_markers, const double* X);

/* Solid-only dynamics, without the fluid (the membrane stretching
 * validation of Sec. 3.2): n_steps of velocity Verlet with viscous damping
 * for every marker, under its body's force (membranes, filaments), the
 * Morse term when set, and the external force f_ext (host [3][M], may be
 * NULL), with mass `mass` per marker:
 *   v' = v + dt/2 (F(X)/m - gamma v);  X += dt v';  v = (v' + dt/2 F(X)/m) / (1 + gamma dt/2).
 * Marker velocities persist across calls and start from rest after
 * set_markers. The lattice is untouched. Errors: E_ARG (dt <= 0, gamma < 0,
 * mass <= 0, n_steps < 0), E_STATE (rigid bodies present: they need the
 * fluid), E_NOMEM. Waits for the GPU. */
int ibm_lbm_solid_steps(ibm_lbm_t* h, int64_t n_steps, double dt, double gamma, double mass, const double* f_ext);

/* Morse excluded volume (Eq. morsePotential, Sec. 2.2) between markers of
 * different membrane or filament bodies: U = D0 (e^{-2 alpha (r - r0)} -
 * 2 e^{-alpha (r - r0)}) for r < rc, added to the marker forces after the
 * bodies' own forces. Periodic axes use the nearest image. Rigid-body
 * markers and tracers do not take part. rc <= 0 switches it off (the
 * default). May be called before or after set_markers. Errors: E_ARG
 * (D0 < 0, alpha <= 0 with rc > 0), E_NOMEM. */
int ibm_lbm_set_morse(ibm_lbm_t* h, double D0, double alpha, double r0, double rc);

/* Advance n_steps coupled steps (order above) and wait for them; the last
 * step also writes the moments of every fluid cell and a FP64 conservation
 * check runs (E_UNSTABLE on a non-finite value or |u| > 0.4). */
int ibm_lbm_step(ibm_lbm_t* h, int64_t n_steps);
/* Same work, enqueued without waiting; ibm_lbm_synchronize waits and
 * returns the status of everything enqueued since the last wait. */
int ibm_lbm_step_async(ibm_lbm_t* h, int64_t n_steps);
int ibm_lbm_synchronize(ibm_lbm_t* h);

/* Moments of the last collision (Eq. rho_u, including half the force
 * density): rho host [N], u host [3][N]; either may be NULL. Solid cells
 * report rho = 0, u = 0. Before any step: the state given to set_lattice. */
int ibm_lbm_get_fields(ibm_lbm_t* h, double* rho, double* u);

/* Markers: X host [3][M] FP64; U (last interpolated velocity, Eq.
 * ibmVelocityInterpret) and F (last marker force) host [3][M] FP64; any
 * may be NULL. */
int ibm_lbm_get_markers(ibm_lbm_t* h, double* X, double* U, double* F);
/* Body records with the current rigid-body state (pose, velocities). */
int ibm_lbm_get_bodies(ibm_lbm_t* h, ibm_lbm_body* bodies, int32_t n_bodies);

/* Diagnostics of the last ibm_lbm_step (FP64 sums over fluid cells of the
 * last collision's moments): out[0] = sum rho, out[1..3] = sum rho u,
 * out[4] = max |u|, out[5] = steps taken since set_lattice,
 * out[6] = fluid cell count, out[7] = 0. */
int ibm_lbm_get_diagnostics(ibm_lbm_t* h, double out[8]);

/* Stage-by-stage execution for verification: runs one stage of the step
 * (IBM_LBM_STAGE_*) on the handle's stream and waits. SPREAD adds into the
 * force density, COLLIDE consumes it and writes the moments of every fluid
 * cell, INTERP clears the force density it consumed and completes the step. */
int ibm_lbm_run_stage(ibm_lbm_t* h, int32_t stage);
/* Overwrite the marker forces (host [3][M]) read by the next SPREAD stage. */
int ibm_lbm_set_marker_forces(ibm_lbm_t* h, const double* F);
/* The spread force density waiting for the next COLLIDE (excluding the
 * uniform body force), host [3][N]; zero after an INTERP stage or a full
 * step. */
int ibm_lbm_get_force_density(ibm_lbm_t* h, double* g);

/* Per-stage timing with CUDA events on the handle's stream (measurement
 * support; no counterpart in the paper beyond its gprof split of the coupling
 * routines, Table tab:timeCoupling). ibm_lbm_set_timing(h, n) with n > 0
 * pre-creates events for n steps and makes the following steps launch their
 * kernels directly (not through graphs) with an event between stages;
 * n = 0 turns timing off. ibm_lbm_get_timing waits for the stream and
 * returns, summed over the timed steps, the milliseconds of out[0] marker
 * forces, out[1] spreading, out[2] collide-stream, out[3] interpolation,
 * out[4] = number of timed steps, out[5] = the part of out[2] spent in
 * odd (neighbour-addressed) AA steps; then resets the sums. */
int ibm_lbm_set_timing(ibm_lbm_t* h, int64_t max_steps);
int ibm_lbm_get_timing(ibm_lbm_t* h, double out[6]);
/* Timing of the production path of membrane suspensions. With on != 0 and
 * timing on, a handle that takes the fused coupling kernel (see
 * ibm_lbm_step) runs its timed steps on that path, with direct launches:
 * each step that launches the fused kernel is timed, out[2] receiving its
 * collision and out[3] the fused kernel (interpolation and advection of the
 * step, marker forces and spreading of the next, Sec. 2.3) with the clear
 * of the touched-tile flags before it; out[0] and out[1] stay zero and
 * out[4] counts these steps. The other steps of the call (the first step's
 * forces and spreading, a step that restores the even AA parity, the last
 * step) run untimed. A handle that does not take the fused path is timed
 * stage by stage as above. on = 0 (the default) restores that for every
 * handle. Returns E_ARG for a NULL handle. */
int ibm_lbm_set_timing_fused(ibm_lbm_t* h, int on);

/* ---------------------------------------------------------------------------
 * Serving: many independent simulations on one GPU with continuous batching.
 * The paper runs one simulation per MPI job; this is the serving pattern of
 * the GB300 build. Cases are submitted at any time and wait in FIFO order
 * until the device-memory budget and a slot allow their admission; every
 * ibm_lbm_server_advance then runs one chunk of steps for all admitted cases
 * together (one batched launch per stage, replayed as a CUDA graph), retires
 * the cases that reached their step count (their results are copied to host
 * memory and their device memory is released) and admits waiting ones. A
 * case's result is the same as running it alone with ibm_lbm_step. Cases use
 * FP32 storage.
 * --------------------------------------------------------------------------- */
typedef struct ibm_lbm_server ibm_lbm_server_t;

typedef struct {
  size_t device_mem_budget;  /* bytes of device memory all admitted cases may hold */
  int32_t max_active;        /* slots (cases advanced together), >= 1 */
  int32_t chunk_steps;       /* steps per advance, even, >= 2 */
  int32_t device;            /* CUDA device ordinal */
} ibm_lbm_server_config;

/* One case: lattice (storage must be IBM_LBM_STORE_F32), initial state
 * (rho0 [N] / u0 [3][N], either NULL for rest), markers, bodies (membranes,
 * rigid bodies; no filaments), mesh (as ibm_lbm_set_markers) and the number
 * of steps to run. All host arrays are copied at submission. */
typedef struct {
  ibm_lbm_config lattice;
  const double* rho0;
  const double* u0;
  const ibm_lbm_mesh* mesh;
  int32_t n_bodies;
  const ibm_lbm_body* bodies;
  int64_t n_markers;
  const double* X;
  int64_t n_steps;
} ibm_lbm_case;

enum { IBM_LBM_CASE_PENDING = 0, IBM_LBM_CASE_RUNNING = 1, IBM_LBM_CASE_DONE = 2 };

/* alloc / stream as for ibm_lbm_create. Errors: E_ARG, E_NOMEM, E_CUDA. */
int ibm_lbm_server_create(const ibm_lbm_server_config* cfg, const ibm_lbm_allocator* alloc, void* stream,
                          ibm_lbm_server_t** out);
int ibm_lbm_server_destroy(ibm_lbm_server_t* s);
/* Queue a case; *id identifies it. E_ARG for an invalid case or one that can
 * never fit the memory budget. */
int ibm_lbm_server_submit(ibm_lbm_server_t* s, const ibm_lbm_case* c, uint64_t* id);
/* Admit what fits, run one chunk (chunk_steps steps; a case stops exactly
 * at its step count), retire finished cases; waits for the GPU. Reports the
 * numbers of running, waiting and finished-not-yet-collected cases (any
 * pointer may be NULL). E_UNSTABLE if a retired case failed its
 * conservation check (its result is still kept). */
int ibm_lbm_server_advance(ibm_lbm_server_t* s, int32_t* n_running, int32_t* n_pending, int32_t* n_done);
/* State (IBM_LBM_CASE_*) and steps completed of a case. */
int ibm_lbm_server_poll(ibm_lbm_server_t* s, uint64_t id, int32_t* state, int64_t* steps_done);
/* Copy a finished case's result into caller memory and forget the case:
 * rho [N], u [3][N] (moments of the last collision, as ibm_lbm_get_fields),
 * X, U [3][M], bodies [n_bodies] (pose of rigid bodies); any pointer may be
 * NULL. E_STATE if the case has not finished. */
int ibm_lbm_server_result(ibm_lbm_server_t* s, uint64_t id, double* rho, double* u, double* X, double* U,
                          ibm_lbm_body* bodies, int32_t n_bodies);
const char* ibm_lbm_server_last_error(const ibm_lbm_server_t* s);

/* Force spreading for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a deployment helper. Some callers
 * cannot call cudaMalloc at all, for example a host framework that has
 * already reserved the GPU's memory for its own pool and forbids further
 * allocations, or a time-critical loop that may not pay allocation latency
 * or synchronisation. This entry point spreads marker forces to the lattice
 * (the same operation as the SPREAD stage of a handle) without a handle and
 * without allocating: it accumulates into a fixed, file-scope device array
 * of IBM_LBM_NOALLOC_MAX_CELLS float4 values (16 MiB), which every GPU that
 * loads this library holds until the process exits.
 *
 * Inputs (device pointers owned by the caller): X [3][M] FP64 marker
 * positions, F [3][M] FP64 marker forces. X is not visible to the host, so
 * it is checked on the device: a marker whose position is not finite or has
 * a coordinate with |x| >= 2^30 (the bound ibm_lbm_set_markers enforces)
 * contributes nothing; non-finite forces give non-finite density. Output: g [3][N] FP64 force
 * density, N = nx*ny*nz, fully overwritten (cells outside every stencil get
 * 0). geometry / tube_radius as in ibm_lbm_config; stream is a cudaStream_t
 * or NULL. The call only enqueues work on the stream and returns; g is ready
 * when the stream reaches that point.
 * Every call looks up the array's device address in the current context
 * (so a device reset by the caller is safe); the first call on a device may
 * load the library's device code there, so make it before any stream
 * capture.
 * Every call shares the one array per device and clears it first, so calls
 * whose work overlaps on the GPU (different streams, host threads) race and
 * must be serialised by the caller.
 * Errors: IBM_LBM_E_ARG if nx*ny*nz > IBM_LBM_NOALLOC_MAX_CELLS, any
 * dimension < 4, M < 0 or M >= 2^31, X or F null with M > 0, g null, an
 * unknown geometry, or geometry 2 (tube) with tube_radius <= 0 (also for any
 * host exception; none crosses this boundary); IBM_LBM_E_CUDA if the
 * address lookup, the clearing of the array or a launch fails. */
#define IBM_LBM_NOALLOC_MAX_CELLS (1 << 20)
int ibm_lbm_spread_noalloc(const double* X, const double* F, int64_t n_markers, int32_t nx, int32_t ny,
                           int32_t nz, int32_t geometry, double tube_radius, double* g, void* stream);

/* The cudaStream_t the handle works on. */
void* ibm_lbm_stream(ibm_lbm_t* h);
/* Bytes of device memory the handle holds. */
size_t ibm_lbm_device_bytes(const ibm_lbm_t* h);
/* Message of the last failed call on h (static text for h == NULL). */
const char* ibm_lbm_last_error(const ibm_lbm_t* h);
const char* ibm_lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IBM_LBM_H */

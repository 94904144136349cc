/*
 * FP64 CPU oracle of the coupled immersed-boundary lattice-Boltzmann step
 * (Tan, Sinno & Diamond, arXiv:1704.04551, Sec. 2.1-2.3).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it. It
 * shares no code, header, table or constant with the CUDA library and must
 * never be linked into it.
 *
 * The oracle is written to be read against the paper, not to be fast:
 * two population arrays with push streaming, plain loops, FP64 throughout.
 *
 * Layouts: cell index idx = x + nx*(y + ny*z); populations [19][N];
 * vectors on the lattice [3][N]; marker arrays [3][M].
 * D3Q19 ordering (shared convention of the public interface, restated here):
 *   0: (0,0,0); 1,2: (+-1,0,0); 3,4: (0,+-1,0); 5,6: (0,0,+-1);
 *   7,8: +-(1,1,0); 9,10: +-(1,-1,0); 11,12: +-(1,0,1); 13,14: +-(1,0,-1);
 *   15,16: +-(0,1,1); 17,18: +-(0,1,-1).
 */
#ifndef IBM_ORACLE_H
#define IBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, ny, nz;
  int32_t geometry;     /* 0 periodic; 1 walls at y=-1/2 and y=ny-1/2; 2 tube along x */
  double tau;           /* BGK relaxation time, nu = (tau - 1/2)/3 (Eq. viscosity) */
  double wall_u[2];     /* x-velocity of the lower / upper y wall (geometry 1) */
  double tube_radius;   /* geometry 2: a cell is solid if its centre is farther from the axis */
  double body_force[3]; /* uniform force density added to the spread density */
} ora_config;

typedef struct {
  int32_t kind;         /* 0 membrane (Eq. membrane-potential), 1 rigid (penalty tether),
                           2 filament (bead chain: Eq. inPlanePotential bonds, Eq.
                           bendingEnergyWorm angles), 3 rigid with the direct FSI
                           forcing of Eq. FSIRigid (kappa = volume per marker) */
  int32_t pad;
  int64_t first, count; /* marker range */
  double kBT_p, k_b, k_l, k_g, k_v;   /* membrane moduli, lattice units */
  double kappa;                        /* rigid: tether stiffness */
  double mass, inertia[3];             /* rigid: mass, principal moments (body frame) */
  double center[3], quat[4];           /* rigid: pose, quaternion (w,x,y,z) body->world */
  double vel[3], omega[3];             /* rigid: velocity, angular velocity (world) */
  double l0;                           /* filament: rest bond length */
} ora_body;

typedef struct ora ora_t;

ora_t* ora_create(const ora_config* cfg);
void ora_destroy(ora_t* o);

/* Lattice: equilibrium initialisation (Sec. 2.1), raw populations. */
void ora_set_equilibrium(ora_t* o, const double* rho, const double* u);
void ora_set_populations(ora_t* o, const double* f);
void ora_get_populations(const ora_t* o, double* f);
/* Moments computed at the last collision (rho [N], u [3][N], incl. g/2). */
void ora_get_fields(const ora_t* o, double* rho, double* u);
/* Force density spread in the last spread stage (excl. the uniform force). */
void ora_get_force_density(const ora_t* o, double* g);
/* Sum over fluid cells of rho and rho*u from the last collision's moments. */
void ora_conserved(const ora_t* o, double out[4]);

/* Markers. The mesh (if any) is the membrane template: tris [T][3]
 * (outward, counter-clockwise), rest shape [3][V]. */
int ora_set_mesh(ora_t* o, int32_t nv, int32_t nt, const int32_t* tris, const double* rest_X);
int ora_set_bodies(ora_t* o, int32_t nb, const ora_body* bodies, int64_t M, const double* X);
void ora_get_markers(const ora_t* o, double* X, double* U, double* F);
/* Overwrite the marker forces [3][M] (consumed by the next spread stage). */
void ora_set_marker_forces(ora_t* o, const double* F);
void ora_get_body(const ora_t* o, int32_t b, ora_body* out);

/* The step, stage by stage, in this order. */
void ora_stage_forces(ora_t* o);          /* marker forces (internal, then Morse; rigid-body update) */
void ora_stage_spread(ora_t* o);          /* Eq. ibmForceSpread */
void ora_stage_collide_stream(ora_t* o);  /* Eq. lbm with BGK and Guo forcing */
void ora_stage_interpolate(ora_t* o);     /* Eq. ibmVelocityInterpret, then X += U */
void ora_step(ora_t* o, int64_t n);
/* Solid-only velocity-Verlet steps with viscous damping (membrane
 * stretching validation, Sec. 3.2); v [3][M] in/out, f_ext [3][M] or NULL. */
void ora_solid_steps(ora_t* o, int64_t n, double dt, double gamma, double mass, const double* f_ext, double* v);

/* Pure helpers, exported for the pins. */
double ora_phi(double r);                                        /* Eq. deltaPhiSimple */
void ora_lattice(int32_t c[19][3], double w[19]);
void ora_equilibrium(double rho, const double u[3], double feq[19]);   /* Eq. BGKequilibrium */
void ora_guo(double tau, const double u[3], const double g[3], double F[19]);
/* Membrane energy of one body at positions X [3][count] (Eqs. inPlanePotential,
 * bendingEnergy, areaEnergy, volumeEnergy), and its analytic forces -dU/dX. */
double ora_membrane_energy(const ora_t* o, int32_t b, const double* X);
void ora_membrane_forces(const ora_t* o, int32_t b, const double* X, double* F);
/* Filament energy of one body at positions X [3][count] (bonds of Eq.
 * inPlanePotential with l_m = 2 l0 and k_p = 1.25 (kBT/p) l0^2; angles of Eq.
 * bendingEnergyWorm with theta0 = pi), and its analytic forces -dU/dX. */
double ora_filament_energy(const ora_t* o, int32_t b, const double* X);
void ora_filament_forces(const ora_t* o, int32_t b, const double* X, double* F);
/* Morse excluded volume (Eq. morsePotential) between markers of different
 * membrane or filament bodies, r < rc; rc <= 0 switches it off. Periodic
 * axes use the nearest image. ora_morse_energy: total over all pairs at
 * positions X [3][M]; ora_morse_forces: -dU/dX [3][M]. */
void ora_set_morse(ora_t* o, double D0, double alpha, double r0, double rc);
double ora_morse_energy(const ora_t* o, const double* X);
void ora_morse_forces(const ora_t* o, const double* X, double* F);
/* Threads of the OpenMP loops (lattice z slabs, markers, bodies; the
 * results do not depend on it); n <= 0 leaves the count unchanged. Returns
 * the count in effect, 1 in a build without OpenMP. */
int ora_set_threads(int n);
/* Rest-state quantities derived from the template: A0, V0, mean l0. */
void ora_mesh_rest(const ora_t* o, double out[3]);
/* Shear modulus of the WLC-POW network (Eq. shearModulus). */
double ora_shear_modulus(double kBT_p, double l0, double x0);

#ifdef __cplusplus
}
#endif
#endif

/*
 * FP64 CPU oracle of the coupled IBM-LBM step of arXiv:1704.04551.
 *
 * TEST INFRASTRUCTURE ONLY (see ibm_oracle.h): used by the tests, the smoke
 * check and the benchmark's CPU baseline; never by the product path.
 *
 * One step, in this order (the paper does not print the order; this is the
 * reading used on both sides):
 *   1. marker forces at X^n: membrane -grad U (Sec. 2.2, Eqs. membrane-potential,
 *      inPlanePotential, bendingEnergy, areaEnergy, volumeEnergy) or, for a
 *      rigid body, a penalty tether to the body's reference points, whose
 *      reaction drives a Newton-Euler update of the body (Sec. 2.3);
 *   2. spreading of the marker forces to the lattice (Eq. ibmForceSpread) with
 *      the 4-point cosine delta (Eq. deltaPhiSimple);
 *   3. BGK collision with Guo forcing and streaming (Eqs. lbm, BGKequilibrium,
 *      rho_u, Guo term), half-way bounce-back at walls;
 *   4. interpolation of the collision-time velocity to the markers
 *      (Eq. ibmVelocityInterpret) and explicit advection X^{n+1} = X^n + U.
 */
#include "ibm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set and weights (Sec. 2.1 cites the standard lattice; the
 * paper does not list them). c_s^2 = 1/3 from Eq. viscosity. */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double WV[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

static int opposite(int i) {
  for (int j = 0; j < Q; ++j)
    if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
  return -1;
}

typedef struct { int32_t a, b, c, d; } edge_t;  /* shared edge a->b, wings c (tri with a->b), d */

struct ora {
  ora_config cfg;
  int64_t N;
  double *f, *fn;    /* [Q][N] */
  double *rho, *u;   /* moments at the last collision */
  double *g;         /* spread force density [3][N] */
  /* markers */
  int64_t M;
  double *X, *U, *F; /* [3][M] */
  double* ref;       /* rigid bodies: body-frame offsets [3][M] */
  int32_t nb;
  ora_body* bodies;
  /* membrane template */
  int32_t nv, nt, ne;
  int32_t* tris;     /* [nt][3] */
  edge_t* edges;
  double *l0, *th0, *At0;
  double A0, V0;
  /* Morse excluded volume */
  double morse_D0, morse_alpha, morse_r0, morse_rc;
};

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static void sub3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

static void quat_matrix(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* geometry                                                                   */
/* ------------------------------------------------------------------------ */
static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Is the lattice node (x,y,z) (unwrapped) solid? Out-of-range coordinates in
 * non-periodic directions are solid. Writes the wrapped index into *idx when
 * the node is fluid. Also returns, through *wall, which y wall (0/1) it is. */
static int node_solid(const ora_t* o, int x, int y, int z, int64_t* idx, int* wall) {
  const ora_config* c = &o->cfg;
  x = wrap(x, c->nx);
  if (wall) *wall = -1;
  if (c->geometry == 0) {
    y = wrap(y, c->ny);
    z = wrap(z, c->nz);
  } else if (c->geometry == 1) {
    z = wrap(z, c->nz);
    if (y < 0) { if (wall) *wall = 0; return 1; }
    if (y >= c->ny) { if (wall) *wall = 1; return 1; }
  } else {
    if (y < 0 || y >= c->ny || z < 0 || z >= c->nz) return 1;
    double yc = 0.5 * (c->ny - 1), zc = 0.5 * (c->nz - 1);
    double dy = y - yc, dz = z - zc;
    if (dy * dy + dz * dz > c->tube_radius * c->tube_radius) return 1;
  }
  if (idx) *idx = x + (int64_t)c->nx * (y + (int64_t)c->ny * z);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* pure helpers                                                               */
/* ------------------------------------------------------------------------ */
double ora_phi(double r) {
  double a = fabs(r);
  if (a > 2.0) return 0.0;
  return 0.25 * (1.0 + cos(M_PI * r / 2.0));
}

void ora_lattice(int32_t c[19][3], double w[19]) {
  for (int i = 0; i < Q; ++i) {
    for (int k = 0; k < 3; ++k) c[i][k] = CV[i][k];
    w[i] = WV[i];
  }
}

void ora_equilibrium(double rho, const double u[3], double feq[19]) {
  double uu = dot3(u, u);
  for (int i = 0; i < Q; ++i) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    feq[i] = WV[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

void ora_guo(double tau, const double u[3], const double g[3], double F[19]) {
  double pre = 1.0 - 1.0 / (2.0 * tau);
  for (int i = 0; i < Q; ++i) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += ((CV[i][k] - u[k]) / CS2 + cu / (CS2 * CS2) * CV[i][k]) * g[k];
    F[i] = pre * WV[i] * s;
  }
}

double ora_shear_modulus(double kBT_p, double l0, double x0) {
  double lm = l0 / x0;
  double kp = kBT_p * l0 * l0 * (1.0 / (4.0 * (1 - x0) * (1 - x0)) - 0.25 + x0);
  return sqrt(3.0) * kBT_p / (4.0 * lm * x0) *
             (x0 / (2.0 * pow(1 - x0, 3)) - 1.0 / (4.0 * (1 - x0) * (1 - x0)) + 0.25) +
         3.0 * sqrt(3.0) * kp / (4.0 * l0 * l0 * l0);
}

/* ------------------------------------------------------------------------ */
/* lifetime                                                                   */
/* ------------------------------------------------------------------------ */
ora_t* ora_create(const ora_config* cfg) {
  ora_t* o = (ora_t*)calloc(1, sizeof(ora_t));
  o->cfg = *cfg;
  o->N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  o->f = (double*)calloc((size_t)Q * o->N, sizeof(double));
  o->fn = (double*)calloc((size_t)Q * o->N, sizeof(double));
  o->rho = (double*)calloc((size_t)o->N, sizeof(double));
  o->u = (double*)calloc((size_t)3 * o->N, sizeof(double));
  o->g = (double*)calloc((size_t)3 * o->N, sizeof(double));
  ora_set_equilibrium(o, NULL, NULL);
  return o;
}

static void free_markers(ora_t* o) {
  free(o->X); free(o->U); free(o->F); free(o->ref); free(o->bodies);
  o->X = o->U = o->F = o->ref = NULL; o->bodies = NULL; o->M = 0; o->nb = 0;
}

static void free_mesh(ora_t* o) {
  free(o->tris); free(o->edges); free(o->l0); free(o->th0); free(o->At0);
  o->tris = NULL; o->edges = NULL; o->l0 = o->th0 = o->At0 = NULL; o->nv = o->nt = o->ne = 0;
}

void ora_destroy(ora_t* o) {
  if (!o) return;
  free(o->f); free(o->fn); free(o->rho); free(o->u); free(o->g);
  free_markers(o); free_mesh(o);
  free(o);
}

/* ------------------------------------------------------------------------ */
/* lattice state                                                              */
/* ------------------------------------------------------------------------ */
void ora_set_equilibrium(ora_t* o, const double* rho, const double* u) {
  const ora_config* c = &o->cfg;
  int64_t N = o->N;
  for (int z = 0; z < c->nz; ++z)
    for (int y = 0; y < c->ny; ++y)
      for (int x = 0; x < c->nx; ++x) {
        int64_t idx = x + (int64_t)c->nx * (y + (int64_t)c->ny * z);
        double r = rho ? rho[idx] : 1.0;
        double v[3] = {u ? u[idx] : 0.0, u ? u[N + idx] : 0.0, u ? u[2 * N + idx] : 0.0};
        double feq[Q];
        int solid = node_solid(o, x, y, z, NULL, NULL);
        ora_equilibrium(r, v, feq);
        for (int i = 0; i < Q; ++i) o->f[i * N + idx] = solid ? 0.0 : feq[i];
        o->rho[idx] = solid ? 0.0 : r;
        for (int k = 0; k < 3; ++k) o->u[k * N + idx] = solid ? 0.0 : v[k];
      }
  memset(o->g, 0, sizeof(double) * 3 * N);
}

void ora_set_populations(ora_t* o, const double* f) {
  memcpy(o->f, f, sizeof(double) * Q * o->N);
}

void ora_get_populations(const ora_t* o, double* f) {
  memcpy(f, o->f, sizeof(double) * Q * o->N);
}

void ora_get_fields(const ora_t* o, double* rho, double* u) {
  if (rho) memcpy(rho, o->rho, sizeof(double) * o->N);
  if (u) memcpy(u, o->u, sizeof(double) * 3 * o->N);
}

void ora_get_force_density(const ora_t* o, double* g) {
  memcpy(g, o->g, sizeof(double) * 3 * o->N);
}

void ora_conserved(const ora_t* o, double out[4]) {
  const ora_config* c = &o->cfg;
  int64_t N = o->N;
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int z = 0; z < c->nz; ++z)
    for (int y = 0; y < c->ny; ++y)
      for (int x = 0; x < c->nx; ++x) {
        int64_t idx;
        if (node_solid(o, x, y, z, &idx, NULL)) continue;
        out[0] += o->rho[idx];
        for (int k = 0; k < 3; ++k) out[1 + k] += o->rho[idx] * o->u[k * N + idx];
      }
}

/* ------------------------------------------------------------------------ */
/* collision + streaming (Eqs. lbm, BGKequilibrium, rho_u, Guo term)          */
/* ------------------------------------------------------------------------ */
void ora_stage_collide_stream(ora_t* o) {
  const ora_config* c = &o->cfg;
  int64_t N = o->N;
  double tau = c->tau;
  memset(o->fn, 0, sizeof(double) * Q * N);
  /* every destination slot has one source cell: the z slabs are independent */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < c->nz; ++z)
    for (int y = 0; y < c->ny; ++y)
      for (int x = 0; x < c->nx; ++x) {
        int64_t idx;
        if (node_solid(o, x, y, z, &idx, NULL)) continue;
        double fi[Q];
        double rho = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          fi[i] = o->f[i * N + idx];
          rho += fi[i];
          for (int k = 0; k < 3; ++k) j[k] += fi[i] * CV[i][k];
        }
        double G[3], u[3];
        for (int k = 0; k < 3; ++k) {
          G[k] = o->g[k * N + idx] + c->body_force[k];
          u[k] = (j[k] + 0.5 * G[k]) / rho;
        }
        o->rho[idx] = rho;
        for (int k = 0; k < 3; ++k) o->u[k * N + idx] = u[k];
        double feq[Q], Fg[Q];
        ora_equilibrium(rho, u, feq);
        ora_guo(tau, u, G, Fg);
        for (int i = 0; i < Q; ++i) {
          double fs = fi[i] - (fi[i] - feq[i]) / tau + Fg[i];
          int64_t t;
          int wall;
          if (node_solid(o, x + CV[i][0], y + CV[i][1], z + CV[i][2], &t, &wall)) {
            /* half-way bounce-back with the moving-wall momentum term */
            double uw = (wall >= 0) ? c->wall_u[wall] : 0.0;
            double cu = CV[i][0] * uw;
            o->fn[opposite(i) * N + idx] = fs - 2.0 * WV[i] * rho * cu / CS2;
          } else {
            o->fn[i * N + t] = fs;
          }
        }
      }
  double* tmp = o->f; o->f = o->fn; o->fn = tmp;
}

/* ------------------------------------------------------------------------ */
/* IBM transfer (Eqs. ibmVelocityInterpret, ibmForceSpread, deltaPhiSimple)   */
/* ------------------------------------------------------------------------ */
void ora_stage_spread(ora_t* o) {
  int64_t N = o->N, M = o->M;
  memset(o->g, 0, sizeof(double) * 3 * N);
  for (int64_t k = 0; k < M; ++k) {
    double X[3] = {o->X[k], o->X[M + k], o->X[2 * M + k]};
    int base[3];
    for (int a = 0; a < 3; ++a) base[a] = (int)floor(X[a]) - 1;
    for (int cz = 0; cz < 4; ++cz)
      for (int cy = 0; cy < 4; ++cy)
        for (int cx = 0; cx < 4; ++cx) {
          int nx_ = base[0] + cx, ny_ = base[1] + cy, nz_ = base[2] + cz;
          int64_t idx;
          if (node_solid(o, nx_, ny_, nz_, &idx, NULL)) continue;
          double d = ora_phi(nx_ - X[0]) * ora_phi(ny_ - X[1]) * ora_phi(nz_ - X[2]);
          for (int a = 0; a < 3; ++a) o->g[a * N + idx] += o->F[a * M + k] * d;
        }
  }
}

void ora_stage_interpolate(ora_t* o) {
  int64_t N = o->N, M = o->M;
  /* markers of direct-forcing rigid bodies follow the body, not the fluid */
  char* fixed = (char*)calloc(M ? M : 1, 1);
  for (int b = 0; b < o->nb; ++b)
    if (o->bodies[b].kind == 3)
      for (int64_t k = o->bodies[b].first; k < o->bodies[b].first + o->bodies[b].count; ++k) fixed[k] = 1;
  /* markers are independent */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < M; ++k) {
    double X[3] = {o->X[k], o->X[M + k], o->X[2 * M + k]};
    int base[3];
    for (int a = 0; a < 3; ++a) base[a] = (int)floor(X[a]) - 1;
    double U[3] = {0, 0, 0};
    for (int cz = 0; cz < 4; ++cz)
      for (int cy = 0; cy < 4; ++cy)
        for (int cx = 0; cx < 4; ++cx) {
          int nx_ = base[0] + cx, ny_ = base[1] + cy, nz_ = base[2] + cz;
          int64_t idx;
          if (node_solid(o, nx_, ny_, nz_, &idx, NULL)) continue;
          double d = ora_phi(nx_ - X[0]) * ora_phi(ny_ - X[1]) * ora_phi(nz_ - X[2]);
          for (int a = 0; a < 3; ++a) U[a] += o->u[a * N + idx] * d;
        }
    for (int a = 0; a < 3; ++a) {
      o->U[a * M + k] = U[a];
      if (!fixed[k]) o->X[a * M + k] = X[a] + U[a];
    }
  }
  free(fixed);
}

/* ------------------------------------------------------------------------ */
/* membrane template                                                          */
/* ------------------------------------------------------------------------ */
static double tri_area(const double* p0, const double* p1, const double* p2) {
  double e1[3], e2[3], n[3];
  sub3(p1, p0, e1); sub3(p2, p0, e2); cross3(e1, e2, n);
  return 0.5 * norm3(n);
}

/* Signed angle between the outward normals of the triangles (a,b,c) and
 * (b,a,d) sharing the edge a-b; positive where the surface is convex. */
static double dihedral(const double* a, const double* b, const double* c, const double* d) {
  double e[3], ca[3], db[3], ab[3], n1[3], n2[3], m[3];
  sub3(b, a, e); sub3(c, a, ca); sub3(a, b, ab); sub3(d, b, db);
  cross3(e, ca, n1); cross3(ab, db, n2);
  cross3(n1, n2, m);
  return atan2(dot3(m, e) / norm3(e), dot3(n1, n2));
}

/* positions of a body's vertex v from an SoA array with stride `stride` */
static void vget(const double* X, int64_t stride, int64_t v, double p[3]) {
  p[0] = X[v]; p[1] = X[stride + v]; p[2] = X[2 * stride + v];
}

int ora_set_mesh(ora_t* o, int32_t nv, int32_t nt, const int32_t* tris, const double* rest_X) {
  free_mesh(o);
  o->nv = nv; o->nt = nt;
  o->tris = (int32_t*)malloc(sizeof(int32_t) * 3 * nt);
  memcpy(o->tris, tris, sizeof(int32_t) * 3 * nt);
  /* edges: adjacency lists per vertex */
  const int MAXD = 32;
  int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * nv * MAXD);
  int32_t* eid = (int32_t*)malloc(sizeof(int32_t) * nv * MAXD);
  int32_t* deg = (int32_t*)calloc(nv, sizeof(int32_t));
  o->edges = (edge_t*)malloc(sizeof(edge_t) * 3 * nt);
  o->ne = 0;
  int bad = 0;
  for (int t = 0; t < nt && !bad; ++t)
    for (int s = 0; s < 3; ++s) {
      int va = tris[3 * t + s], vb = tris[3 * t + (s + 1) % 3], vc = tris[3 * t + (s + 2) % 3];
      int lo = va < vb ? va : vb, hi = va < vb ? vb : va;
      int found = -1;
      for (int q = 0; q < deg[lo]; ++q)
        if (nbr[lo * MAXD + q] == hi) found = eid[lo * MAXD + q];
      if (found < 0) {
        if (deg[lo] >= MAXD) { bad = 1; break; }
        edge_t e = {va, vb, vc, -1};
        o->edges[o->ne] = e;
        nbr[lo * MAXD + deg[lo]] = hi;
        eid[lo * MAXD + deg[lo]] = o->ne;
        deg[lo]++;
        o->ne++;
      } else {
        edge_t* e = &o->edges[found];
        if (e->d >= 0 || e->a != vb || e->b != va) { bad = 1; break; }
        e->d = vc;
      }
    }
  for (int e = 0; e < o->ne && !bad; ++e)
    if (o->edges[e].d < 0) bad = 1;
  free(nbr); free(eid); free(deg);
  if (bad) { free_mesh(o); return -1; }
  /* rest state */
  o->l0 = (double*)malloc(sizeof(double) * o->ne);
  o->th0 = (double*)malloc(sizeof(double) * o->ne);
  o->At0 = (double*)malloc(sizeof(double) * nt);
  for (int e = 0; e < o->ne; ++e) {
    double a[3], b[3], c[3], d[3], ab[3];
    vget(rest_X, nv, o->edges[e].a, a); vget(rest_X, nv, o->edges[e].b, b);
    vget(rest_X, nv, o->edges[e].c, c); vget(rest_X, nv, o->edges[e].d, d);
    sub3(b, a, ab);
    o->l0[e] = norm3(ab);
    o->th0[e] = dihedral(a, b, c, d);
  }
  o->A0 = 0.0; o->V0 = 0.0;
  for (int t = 0; t < nt; ++t) {
    double p0[3], p1[3], p2[3], x12[3];
    vget(rest_X, nv, tris[3 * t], p0); vget(rest_X, nv, tris[3 * t + 1], p1); vget(rest_X, nv, tris[3 * t + 2], p2);
    o->At0[t] = tri_area(p0, p1, p2);
    o->A0 += o->At0[t];
    cross3(p1, p2, x12);
    o->V0 += dot3(p0, x12) / 6.0;
  }
  return 0;
}

void ora_mesh_rest(const ora_t* o, double out[3]) {
  double s = 0.0;
  for (int e = 0; e < o->ne; ++e) s += o->l0[e];
  out[0] = o->A0; out[1] = o->V0; out[2] = o->ne ? s / o->ne : 0.0;
}

/* total area and volume of a body at positions X (SoA, stride nv) */
static void area_volume(const ora_t* o, const double* X, double* A, double* V) {
  *A = 0.0; *V = 0.0;
  for (int t = 0; t < o->nt; ++t) {
    double p0[3], p1[3], p2[3], x12[3];
    vget(X, o->nv, o->tris[3 * t], p0); vget(X, o->nv, o->tris[3 * t + 1], p1); vget(X, o->nv, o->tris[3 * t + 2], p2);
    *A += tri_area(p0, p1, p2);
    cross3(p1, p2, x12);
    *V += dot3(p0, x12) / 6.0;
  }
}

double ora_membrane_energy(const ora_t* o, int32_t bi, const double* X) {
  const ora_body* b = &o->bodies[bi];
  double U = 0.0;
  for (int e = 0; e < o->ne; ++e) {
    double a[3], bb[3], c[3], d[3], ab[3];
    vget(X, o->nv, o->edges[e].a, a); vget(X, o->nv, o->edges[e].b, bb);
    vget(X, o->nv, o->edges[e].c, c); vget(X, o->nv, o->edges[e].d, d);
    sub3(bb, a, ab);
    double l = norm3(ab), l0 = o->l0[e], lm = 2.0 * l0, x = l / lm;
    double kp = 1.25 * b->kBT_p * l0 * l0;  /* zero net bond force at x = 1/2 */
    U += b->kBT_p * lm / 4.0 * (3 * x * x - 2 * x * x * x) / (1 - x) + kp / l;
    U += b->k_b * (1.0 - cos(dihedral(a, bb, c, d) - o->th0[e]));
  }
  double A, V;
  area_volume(o, X, &A, &V);
  for (int t = 0; t < o->nt; ++t) {
    double p0[3], p1[3], p2[3];
    vget(X, o->nv, o->tris[3 * t], p0); vget(X, o->nv, o->tris[3 * t + 1], p1); vget(X, o->nv, o->tris[3 * t + 2], p2);
    double At = tri_area(p0, p1, p2);
    U += b->k_l * (At - o->At0[t]) * (At - o->At0[t]) / (2.0 * o->At0[t]);
  }
  U += b->k_g * (A - o->A0) * (A - o->A0) / (2.0 * o->A0);
  U += b->k_v * (V - o->V0) * (V - o->V0) / (2.0 * o->V0);
  return U;
}

static void add3(double* F, int64_t stride, int64_t v, const double g[3], double s) {
  F[v] += s * g[0]; F[stride + v] += s * g[1]; F[2 * stride + v] += s * g[2];
}

void ora_membrane_forces(const ora_t* o, int32_t bi, const double* X, double* F) {
  const ora_body* b = &o->bodies[bi];
  int64_t nv = o->nv;
  memset(F, 0, sizeof(double) * 3 * nv);
  for (int e = 0; e < o->ne; ++e) {
    const edge_t* E = &o->edges[e];
    double a[3], bb[3], c[3], d[3], ev[3];
    vget(X, nv, E->a, a); vget(X, nv, E->b, bb); vget(X, nv, E->c, c); vget(X, nv, E->d, d);
    sub3(bb, a, ev);
    /* stretching: WLC + POW (Eq. inPlanePotential), dU/dl along the bond */
    double l = norm3(ev), l0 = o->l0[e], lm = 2.0 * l0, x = l / lm;
    double kp = 1.25 * b->kBT_p * l0 * l0;
    double dUdl = b->kBT_p * (1.0 / (4.0 * (1 - x) * (1 - x)) - 0.25 + x) - kp / (l * l);
    add3(F, nv, E->a, ev, dUdl / l);   /* -dU/dl * (a-b)/l = +dU/dl * (b-a)/l */
    add3(F, nv, E->b, ev, -dUdl / l);
    /* bending (Eq. bendingEnergy): F_v = -k_b sin(theta-theta0) dtheta/dv */
    double ca[3], db[3], ab[3], n1[3], n2[3];
    sub3(c, a, ca); sub3(a, bb, ab); sub3(d, bb, db);
    cross3(ev, ca, n1); cross3(ab, db, n2);
    double L2 = dot3(ev, ev), L = sqrt(L2);
    double n1s = dot3(n1, n1), n2s = dot3(n2, n2);
    double da[3];
    sub3(d, a, da);
    double t1 = dot3(ca, ev) / L2, t2 = dot3(da, ev) / L2;
    double s = b->k_b * sin(dihedral(a, bb, c, d) - o->th0[e]);
    double gc[3], gd[3], ga[3], gb[3];
    for (int k = 0; k < 3; ++k) {
      gc[k] = -L * n1[k] / n1s;
      gd[k] = -L * n2[k] / n2s;
      ga[k] = -(1.0 - t1) * gc[k] - (1.0 - t2) * gd[k];
      gb[k] = -t1 * gc[k] - t2 * gd[k];
    }
    add3(F, nv, E->a, ga, -s); add3(F, nv, E->b, gb, -s);
    add3(F, nv, E->c, gc, -s); add3(F, nv, E->d, gd, -s);
  }
  double A, V;
  area_volume(o, X, &A, &V);
  double cg = b->k_g * (A - o->A0) / o->A0;
  double cv = b->k_v * (V - o->V0) / o->V0;
  for (int t = 0; t < o->nt; ++t) {
    int32_t v[3] = {o->tris[3 * t], o->tris[3 * t + 1], o->tris[3 * t + 2]};
    double p[3][3];
    for (int s = 0; s < 3; ++s) vget(X, nv, v[s], p[s]);
    double e1[3], e2[3], N[3];
    sub3(p[1], p[0], e1); sub3(p[2], p[0], e2); cross3(e1, e2, N);
    double nN = norm3(N), At = 0.5 * nN;
    double nh[3] = {N[0] / nN, N[1] / nN, N[2] / nN};
    /* Eq. areaEnergy: local and global terms share dA_t/dx_v = 1/2 n x (x_{v+2} - x_{v+1}) */
    double coef = b->k_l * (At - o->At0[t]) / o->At0[t] + cg;
    for (int s = 0; s < 3; ++s) {
      double opp[3], gA[3], gV[3];
      sub3(p[(s + 2) % 3], p[(s + 1) % 3], opp);
      cross3(nh, opp, gA);
      add3(F, nv, v[s], gA, -0.5 * coef);
      /* Eq. volumeEnergy: dV/dx_v = (x_{v+1} x x_{v+2}) / 6 */
      cross3(p[(s + 1) % 3], p[(s + 2) % 3], gV);
      add3(F, nv, v[s], gV, -cv / 6.0);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* markers and bodies                                                         */
/* ------------------------------------------------------------------------ */
int ora_set_bodies(ora_t* o, int32_t nb, const ora_body* bodies, int64_t M, const double* X) {
  free_markers(o);
  o->M = M; o->nb = nb;
  o->X = (double*)malloc(sizeof(double) * 3 * (M ? M : 1));
  o->U = (double*)calloc(3 * (M ? M : 1), sizeof(double));
  o->F = (double*)calloc(3 * (M ? M : 1), sizeof(double));
  o->ref = (double*)calloc(3 * (M ? M : 1), sizeof(double));
  o->bodies = (ora_body*)malloc(sizeof(ora_body) * (nb ? nb : 1));
  if (M) memcpy(o->X, X, sizeof(double) * 3 * M);
  if (nb) memcpy(o->bodies, bodies, sizeof(ora_body) * nb);
  for (int b = 0; b < nb; ++b) {
    const ora_body* B = &o->bodies[b];
    if (B->first < 0 || B->count < 0 || B->first + B->count > M) return -1;
    if (B->kind == 0 && B->count != o->nv) return -2;
    if (B->kind == 2 && (B->count < 2 || !(B->l0 > 0.0))) return -3;
    if (B->kind == 1 || B->kind == 3) {
      double R[3][3];
      quat_matrix(B->quat, R);
      for (int64_t k = B->first; k < B->first + B->count; ++k) {
        double d[3] = {X[k] - B->center[0], X[M + k] - B->center[1], X[2 * M + k] - B->center[2]};
        for (int a = 0; a < 3; ++a)
          o->ref[a * M + k] = R[0][a] * d[0] + R[1][a] * d[1] + R[2][a] * d[2];
      }
    }
  }
  return 0;
}

void ora_get_markers(const ora_t* o, double* X, double* U, double* F) {
  if (X) memcpy(X, o->X, sizeof(double) * 3 * o->M);
  if (U) memcpy(U, o->U, sizeof(double) * 3 * o->M);
  if (F) memcpy(F, o->F, sizeof(double) * 3 * o->M);
}

void ora_set_marker_forces(ora_t* o, const double* F) {
  if (o->M) memcpy(o->F, F, sizeof(double) * 3 * o->M);
}

void ora_get_body(const ora_t* o, int32_t b, ora_body* out) { *out = o->bodies[b]; }

/* One explicit Newton-Euler step of a rigid body from its total force FB and
 * torque TB (world frame, about the centre); R the rotation before the step. */
static void rigid_update(ora_body* B, double R[3][3], const double FB[3], const double TB[3]) {
  for (int a = 0; a < 3; ++a) {
    B->vel[a] += FB[a] / B->mass;
    B->center[a] += B->vel[a];
  }
  double wb[3], tb[3], Iw[3], gyro[3];
  for (int a = 0; a < 3; ++a) {
    wb[a] = R[0][a] * B->omega[0] + R[1][a] * B->omega[1] + R[2][a] * B->omega[2];
    tb[a] = R[0][a] * TB[0] + R[1][a] * TB[1] + R[2][a] * TB[2];
  }
  for (int a = 0; a < 3; ++a) Iw[a] = B->inertia[a] * wb[a];
  cross3(wb, Iw, gyro);
  for (int a = 0; a < 3; ++a) wb[a] += (tb[a] - gyro[a]) / B->inertia[a];
  for (int a = 0; a < 3; ++a) B->omega[a] = R[a][0] * wb[0] + R[a][1] * wb[1] + R[a][2] * wb[2];
  /* dq = 1/2 (0, omega) * q, then renormalise */
  double w = B->quat[0], x = B->quat[1], y = B->quat[2], z = B->quat[3];
  double ox = B->omega[0], oy = B->omega[1], oz = B->omega[2];
  double dq[4] = {0.5 * (-ox * x - oy * y - oz * z), 0.5 * (ox * w + oy * z - oz * y),
                  0.5 * (-ox * z + oy * w + oz * x), 0.5 * (ox * y - oy * x + oz * w)};
  double n = 0.0;
  for (int a = 0; a < 4; ++a) { B->quat[a] += dq[a]; n += B->quat[a] * B->quat[a]; }
  n = sqrt(n);
  for (int a = 0; a < 4; ++a) B->quat[a] /= n;
}

/* Rigid body: tether each marker to its body-fixed reference point (penalty
 * reading of the rigid FSI coupling, Sec. 2.3); the reaction gives the
 * body's force and torque, then one explicit Newton-Euler step. */
static void rigid_forces(ora_t* o, ora_body* B) {
  int64_t M = o->M;
  double R[3][3];
  quat_matrix(B->quat, R);
  double FB[3] = {0, 0, 0}, TB[3] = {0, 0, 0};
  for (int64_t k = B->first; k < B->first + B->count; ++k) {
    double r[3] = {o->ref[k], o->ref[M + k], o->ref[2 * M + k]};
    double rw[3], d[3], f[3], t[3];
    for (int a = 0; a < 3; ++a) rw[a] = R[a][0] * r[0] + R[a][1] * r[1] + R[a][2] * r[2];
    for (int a = 0; a < 3; ++a) {
      d[a] = o->X[a * M + k] - (B->center[a] + rw[a]);
      o->F[a * M + k] = -B->kappa * d[a];
      f[a] = B->kappa * d[a];
      FB[a] += f[a];
    }
    cross3(rw, f, t);
    for (int a = 0; a < 3; ++a) TB[a] += t[a];
  }
  rigid_update(B, R, FB, TB);
}

/* Rigid body with the paper's direct FSI forcing (Eq. FSIRigid): the force
 * density on the solid at a marker is rho_f (u(X) - U(X)) / dt, u the fluid
 * velocity interpolated at the marker (Eq. ibmVelocityInterpret, the last
 * interpolation), U = V + omega x (X - C) the body's velocity there; as a
 * nodal force it is weighted by the volume the marker stands for, kappa
 * (rho_f = 1, dt = 1). The fluid receives the opposite force; the sum gives
 * the body's force and torque, one explicit Newton-Euler step, and the
 * markers are moved rigidly to the new pose. */
static void rigid_direct_forces(ora_t* o, ora_body* B) {
  int64_t M = o->M;
  double R[3][3];
  quat_matrix(B->quat, R);
  double FB[3] = {0, 0, 0}, TB[3] = {0, 0, 0};
  for (int64_t k = B->first; k < B->first + B->count; ++k) {
    double r[3] = {o->ref[k], o->ref[M + k], o->ref[2 * M + k]};
    double rw[3], us[3], f[3], t[3];
    for (int a = 0; a < 3; ++a) rw[a] = R[a][0] * r[0] + R[a][1] * r[1] + R[a][2] * r[2];
    cross3(B->omega, rw, us);
    for (int a = 0; a < 3; ++a) {
      us[a] += B->vel[a];
      f[a] = B->kappa * (o->U[a * M + k] - us[a]);
      o->F[a * M + k] = -f[a];
      FB[a] += f[a];
    }
    cross3(rw, f, t);
    for (int a = 0; a < 3; ++a) TB[a] += t[a];
  }
  rigid_update(B, R, FB, TB);
  quat_matrix(B->quat, R);
  for (int64_t k = B->first; k < B->first + B->count; ++k) {
    double r[3] = {o->ref[k], o->ref[M + k], o->ref[2 * M + k]};
    for (int a = 0; a < 3; ++a)
      o->X[a * M + k] = B->center[a] + R[a][0] * r[0] + R[a][1] * r[1] + R[a][2] * r[2];
  }
}

/* ------------------------------------------------------------------------ */
/* filaments (Sec. 2.2, polymer particles)                                    */
/* ------------------------------------------------------------------------ */
/* Bond energy of Eq. inPlanePotential for one bond of length l, rest l0:
 * WLC with x = l / l_m, l_m = 2 l0, plus the POW term k_p / l with
 * k_p = 1.25 (kBT/p) l0^2 (zero bond force at l = l0). */
static double bond_energy(double kBT_p, double l0, double l) {
  const double lm = 2.0 * l0, x = l / lm, kp = 1.25 * kBT_p * l0 * l0;
  return kBT_p * lm / 4.0 * (3.0 * x * x - 2.0 * x * x * x) / (1.0 - x) + kp / l;
}
static double bond_dUdl(double kBT_p, double l0, double l) {
  const double x = l / (2.0 * l0), kp = 1.25 * kBT_p * l0 * l0;
  return kBT_p * (0.25 / ((1.0 - x) * (1.0 - x)) - 0.25 + x) - kp / (l * l);
}

/* angle at bead j between the bonds to its neighbours, in [0, pi] */
static double bead_angle(const double* a, const double* j, const double* c) {
  double u[3], v[3], w[3];
  sub3(a, j, u);
  sub3(c, j, v);
  cross3(u, v, w);
  return atan2(norm3(w), dot3(u, v));
}

double ora_filament_energy(const ora_t* o, int32_t bi, const double* X) {
  const ora_body* B = &o->bodies[bi];
  const int64_t n = B->count;
  double U = 0.0;
  for (int64_t j = 0; j + 1 < n; ++j) {
    double p[3], q[3], d[3];
    vget(X, n, j, p);
    vget(X, n, j + 1, q);
    sub3(q, p, d);
    U += bond_energy(B->kBT_p, B->l0, norm3(d));
  }
  for (int64_t j = 1; j + 1 < n; ++j) {
    double a[3], b[3], c[3];
    vget(X, n, j - 1, a);
    vget(X, n, j, b);
    vget(X, n, j + 1, c);
    const double dth = bead_angle(a, b, c) - M_PI;  /* theta0 = 180 degrees */
    U += B->k_b * dth * dth;
  }
  return U;
}

void ora_filament_forces(const ora_t* o, int32_t bi, const double* X, double* F) {
  const ora_body* B = &o->bodies[bi];
  const int64_t n = B->count;
  memset(F, 0, sizeof(double) * 3 * n);
  for (int64_t j = 0; j + 1 < n; ++j) {
    double p[3], q[3], d[3];
    vget(X, n, j, p);
    vget(X, n, j + 1, q);
    sub3(q, p, d);
    const double l = norm3(d), s = bond_dUdl(B->kBT_p, B->l0, l) / l;
    add3(F, n, j, d, s);    /* -dU/dp = dU/dl (q - p)/l */
    add3(F, n, j + 1, d, -s);
  }
  for (int64_t j = 1; j + 1 < n; ++j) {
    /* U = k_b (theta - pi)^2, cos(theta) = u.v / (|u||v|), u = a - b, v = c - b;
     * dU/dcos = 2 k_b (pi - theta) / sin(theta), whose limit at theta = pi is 2 k_b */
    double a[3], b[3], c[3], u[3], v[3], w[3];
    vget(X, n, j - 1, a);
    vget(X, n, j, b);
    vget(X, n, j + 1, c);
    sub3(a, b, u);
    sub3(c, b, v);
    cross3(u, v, w);
    const double lu = norm3(u), lv = norm3(v);
    const double sn = norm3(w) / (lu * lv), cs = dot3(u, v) / (lu * lv);
    const double phi = M_PI - atan2(norm3(w), dot3(u, v));
    const double ratio = sn > 1e-12 ? phi / sn : 1.0 + phi * phi / 6.0;
    const double g = 2.0 * B->k_b * ratio;
    double fa[3], fc[3];
    for (int k = 0; k < 3; ++k) {
      fa[k] = -g * (v[k] / (lu * lv) - cs * u[k] / (lu * lu));
      fc[k] = -g * (u[k] / (lu * lv) - cs * v[k] / (lv * lv));
    }
    add3(F, n, j - 1, fa, 1.0);
    add3(F, n, j + 1, fc, 1.0);
    add3(F, n, j, fa, -1.0);
    add3(F, n, j, fc, -1.0);
  }
}

/* ------------------------------------------------------------------------ */
/* Morse excluded volume between bodies (Eq. morsePotential)                  */
/* ------------------------------------------------------------------------ */
void ora_set_morse(ora_t* o, double D0, double alpha, double r0, double rc) {
  o->morse_D0 = D0; o->morse_alpha = alpha; o->morse_r0 = r0; o->morse_rc = rc;
}

/* body of each marker taking part (membranes, filaments), -1 otherwise */
static int32_t* morse_owner(const ora_t* o) {
  int32_t* own = (int32_t*)malloc(sizeof(int32_t) * (o->M ? o->M : 1));
  for (int64_t k = 0; k < o->M; ++k) own[k] = -1;
  for (int b = 0; b < o->nb; ++b)
    if (o->bodies[b].kind == 0 || o->bodies[b].kind == 2)
      for (int64_t k = o->bodies[b].first; k < o->bodies[b].first + o->bodies[b].count; ++k) own[k] = b;
  return own;
}

/* nearest-image separation X_k - X_j on the periodic axes of the geometry */
static void separation(const ora_t* o, const double* X, int64_t k, int64_t j, double d[3]) {
  const int64_t M = o->M;
  const int n[3] = {o->cfg.nx, o->cfg.ny, o->cfg.nz};
  const int periodic[3] = {1, o->cfg.geometry == 0, o->cfg.geometry != 2};
  for (int a = 0; a < 3; ++a) {
    d[a] = X[a * M + k] - X[a * M + j];
    if (periodic[a]) d[a] -= n[a] * floor(d[a] / n[a] + 0.5);
  }
}

double ora_morse_energy(const ora_t* o, const double* X) {
  if (!(o->morse_rc > 0.0)) return 0.0;
  int32_t* own = morse_owner(o);
  double U = 0.0;
  for (int64_t k = 0; k < o->M; ++k)
    for (int64_t j = k + 1; j < o->M; ++j) {
      if (own[k] < 0 || own[j] < 0 || own[k] == own[j]) continue;
      double d[3];
      separation(o, X, k, j, d);
      const double r = norm3(d);
      if (r >= o->morse_rc) continue;
      const double e = exp(-o->morse_alpha * (r - o->morse_r0));
      U += o->morse_D0 * (e * e - 2.0 * e);
    }
  free(own);
  return U;
}

void ora_morse_forces(const ora_t* o, const double* X, double* F) {
  const int64_t M = o->M;
  memset(F, 0, sizeof(double) * 3 * (M ? M : 1));
  if (!(o->morse_rc > 0.0)) return;
  int32_t* own = morse_owner(o);
  for (int64_t k = 0; k < M; ++k)
    for (int64_t j = k + 1; j < M; ++j) {
      if (own[k] < 0 || own[j] < 0 || own[k] == own[j]) continue;
      double d[3];
      separation(o, X, k, j, d);
      const double r = norm3(d);
      if (r >= o->morse_rc) continue;
      /* dU/dr = 2 alpha D0 (e - e^2), e = exp(-alpha (r - r0)); F_k = -dU/dr d/r */
      const double e = exp(-o->morse_alpha * (r - o->morse_r0));
      const double s = -2.0 * o->morse_alpha * o->morse_D0 * (e - e * e) / r;
      for (int a = 0; a < 3; ++a) {
        F[a * M + k] += s * d[a];
        F[a * M + j] -= s * d[a];
      }
    }
  free(own);
}

void ora_stage_forces(ora_t* o) {
  int64_t M = o->M;
  memset(o->F, 0, sizeof(double) * 3 * (M ? M : 1));
  /* each body writes only its own markers' forces and its own record */
#pragma omp parallel for schedule(dynamic, 4)
  for (int b = 0; b < o->nb; ++b) {
    ora_body* B = &o->bodies[b];
    if (B->kind == 1) {
      rigid_forces(o, B);
    } else if (B->kind == 3) {
      rigid_direct_forces(o, B);
    } else if (B->kind == 0) {
      int64_t nv = o->nv;
      double* Xb = (double*)malloc(sizeof(double) * 3 * nv);
      double* Fb = (double*)malloc(sizeof(double) * 3 * nv);
      for (int a = 0; a < 3; ++a) memcpy(Xb + a * nv, o->X + a * M + B->first, sizeof(double) * nv);
      ora_membrane_forces(o, b, Xb, Fb);
      for (int a = 0; a < 3; ++a) memcpy(o->F + a * M + B->first, Fb + a * nv, sizeof(double) * nv);
      free(Xb); free(Fb);
    } else if (B->kind == 2) {
      const int64_t n = B->count;
      double* Xb = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
      double* Fb = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
      for (int a = 0; a < 3; ++a) memcpy(Xb + a * n, o->X + a * M + B->first, sizeof(double) * n);
      ora_filament_forces(o, b, Xb, Fb);
      for (int a = 0; a < 3; ++a) memcpy(o->F + a * M + B->first, Fb + a * n, sizeof(double) * n);
      free(Xb); free(Fb);
    }
  }
  if (o->morse_rc > 0.0 && M > 0) {
    double* Fm = (double*)malloc(sizeof(double) * 3 * M);
    ora_morse_forces(o, o->X, Fm);
    for (int64_t i = 0; i < 3 * M; ++i) o->F[i] += Fm[i];
    free(Fm);
  }
}

/* Solid-only dynamics (the membrane stretching validation of Sec. 3.2): the
 * markers move under their bodies' forces, the Morse term and an external
 * force f_ext [3][M], with mass m per marker and viscous damping gamma, by
 * velocity Verlet (the damping taken half explicitly in the first half-kick
 * and half implicitly in the second):
 *   v' = v + dt/2 (F(X)/m - gamma v);  X += dt v';
 *   v  = (v' + dt/2 F(X)/m) / (1 + gamma dt/2).
 * v [3][M] is kept by the caller (zero to start from rest). No fluid. */
void ora_solid_steps(ora_t* o, int64_t n, double dt, double gamma, double mass, const double* f_ext, double* v) {
  const int64_t M = o->M;
  for (int64_t s = 0; s < n; ++s) {
    ora_stage_forces(o);
    for (int64_t i = 0; i < 3 * M; ++i) {
      const double F = o->F[i] + (f_ext ? f_ext[i] : 0.0);
      v[i] += 0.5 * dt * (F / mass - gamma * v[i]);
      o->X[i] += dt * v[i];
    }
    ora_stage_forces(o);
    for (int64_t i = 0; i < 3 * M; ++i) {
      const double F = o->F[i] + (f_ext ? f_ext[i] : 0.0);
      v[i] = (v[i] + 0.5 * dt * F / mass) / (1.0 + 0.5 * gamma * dt);
    }
  }
}

int ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void ora_step(ora_t* o, int64_t n) {
  for (int64_t s = 0; s < n; ++s) {
    ora_stage_forces(o);
    ora_stage_spread(o);
    ora_stage_collide_stream(o);
    ora_stage_interpolate(o);
  }
}

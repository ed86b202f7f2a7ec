/*
 * lbm_oracle.c -- FP64 CPU reference of the consistent VANSE lattice Boltzmann
 * scheme of Bukreev, Simonis, Kummerlaender, Jessberger and Krause,
 * "Consistent lattice Boltzmann methods for the volume averaged Navier-Stokes
 * equations" (arXiv 2208.09267).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library; it keeps its own copy of every constant.
 *
 * It is written to be read against the paper, not to be fast:
 *   - two population arrays (old/new), array-of-structures f[cell*Q + i];
 *   - push streaming: the post-collision value of cell x travels to x + xi_i
 *     (left-hand side of the LBE, Sec. 2.2 eq. (lbe));
 *   - every quantity of Sec. 2.2 is formed in the order the paper defines it:
 *     zeroth/first moments, quadrature of the volume fraction (eq. (quad),
 *     Table "weights"), effective density (eq. (density)), pressure-correction
 *     force (eq. (pressForce)) with its central-difference gradient, velocity
 *     with the Guo half-force shift (eq. (velocity)), the equilibrium with the
 *     zeroth moment in place of rho*phi (eq. (feq)), the Guo forcing term, and
 *     the BGK update (eq. (lbe)).
 *
 * Readings of the paper that this file takes (all lattice units,
 * dx = dt = 1, c_s^2 = 1/3):
 *   R1  Direction order inside a group of Tables "latt_par"/"latt_3d" is not
 *       given; opposite directions are stored next to each other:
 *       rest, +x,-x,+y,-y,+z,-z, face diagonals in opposite pairs, corners in
 *       opposite pairs.
 *   R2  Pressure is the deviation p = c_s^2 (rho~ - rho0); the pressure
 *       correction force uses the full effective density,
 *       F_PC = c_s^2 rho~ grad(phi) (eq. (pressForce)).
 *   R3  The quadrature (eq. (quad)) runs over the face neighbours of the
 *       axes selected by the caller (quad_axes) with the weights of Table
 *       "weights" for quad_dim = number of those axes; the gradient of
 *       eq. (pressForce) is taken on every lattice axis.
 *   R4  The volume fraction varies in time through a caller-supplied pair
 *       (phi_ref, d_t phi): phi_n = phi_ref + (n - n_ref) d_t phi.  The same
 *       holds for the optional per-cell force field.  Between refreshes this
 *       is a linear extrapolation; with a refresh each step it is exact.
 *   R5  External force density g (uniform) and the optional field enter the
 *       force sum directly, beside F_PC, as F_MMS does in Sec. 3.
 *   R6  Walls (not in the paper): the first and last layer along each axis
 *       flagged in `walls` is solid; halfway bounce-back sends a population
 *       that would enter a solid cell back to its origin in the opposite
 *       direction.  Solid cells are never updated.
 *   R7  D3Q19 (not in the paper) uses the textbook weights 1/3, 1/18, 1/36.
 *   R8  quad_dim = -1 selects the pointwise density rho~ = M0 / phi(x)
 *       (varpi_0 = 1, varpi_{i!=0} = 0 in eq. (quad)): the zeroth-moment
 *       interpretation the introduction attributes to the earlier scheme of
 *       Zhang et al., kept for the comparison of Sec. 1's claim that it
 *       misses the pressure.  Everything else is the same update.
 *   R9  Phase-interaction drag (Sec. 2.2 lists drag among the forces F_k of
 *       the force sum; the Conclusion names interaction forces as the next
 *       step).  Ergun-type law of a fixed bed of particles of diameter d:
 *       F_D = -(b_lin + b_q |u|) u, b_lin = rho~ c1 (1 - phi)^2 nu / (phi d^2),
 *       b_q = rho~ c2 (1 - phi) / d (Ergun: c1 = 150, c2 = 1.75), phi and
 *       rho~ of the cell at time n, nu = (tau - 1/2)/3.  It is taken
 *       implicitly in eq. (velocity) (see orc_cell_macro), so u and the
 *       force sum stay consistent with the Guo scheme.
 *   R10 Smagorinsky large-eddy closure (the Conclusion names LES as a use of
 *       the scheme): a local relaxation time from the non-equilibrium
 *       momentum flux, tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 Q / M0))/2,
 *       Q = |Pi^neq|, Pi^neq_ab = sum_i xi_ia xi_ib (f_i - f_i^eq): the root
 *       of nu_eff = nu + (C Delta)^2 |S| with |S| = sqrt(2 S:S) from
 *       S = -Pi^neq / (2 c_s^2 M0 tau_eff), Delta = 1.  The Guo term uses
 *       1 - 1/(2 tau_eff).  C = 0 is the BGK update unchanged.
 *
 * Canonical evaluation order.  Every sum runs in ascending index order and
 * starts from 0.0; products are evaluated left to right as written below.
 * The FP64 GPU kernel follows the same order so that the two agree bit for
 * bit; this file is compiled with -ffp-contract=off so that no multiply-add
 * is fused.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Velocity sets (Table "latt_par" for D2Q9, Table "latt_3d" for D3Q27;      */
/* D3Q19 and D1Q3 from the textbook the paper cites for the CE analysis;     */
/* Sec. 2.2 names one-dimensional stencils beside the 2D and 3D ones).       */
/* ------------------------------------------------------------------------ */

#define ORC_MAXQ 27

typedef struct {
  int d;                 /* spatial dimension */
  int q;                 /* number of populations */
  int c[ORC_MAXQ][3];    /* xi_i */
  double w[ORC_MAXQ];    /* w_i */
  int opp[ORC_MAXQ];     /* index of -xi_i */
} orc_vset;

static const int ORC_D1Q3_C[3][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}};

static const int ORC_D2Q9_C[9][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

static const int ORC_D3Q27_C[27][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

/* Build the velocity set; returns 0 on success. */
static int orc_make_vset(int lattice, orc_vset *v) {
  int i, a;
  memset(v, 0, sizeof(*v));
  if (lattice == 0) { /* D2Q9, Table "latt_par": 4/9, 1/9, 1/36 */
    v->d = 2;
    v->q = 9;
    for (i = 0; i < 9; ++i) {
      for (a = 0; a < 3; ++a) v->c[i][a] = ORC_D2Q9_C[i][a];
      v->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else if (lattice == 1) { /* D3Q19: rest, 6 axes, 12 face diagonals */
    v->d = 3;
    v->q = 19;
    for (i = 0; i < 19; ++i) {
      for (a = 0; a < 3; ++a) v->c[i][a] = ORC_D3Q27_C[i][a];
      v->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
  } else if (lattice == 2) { /* D3Q27, Table "latt_3d": 8/27, 2/27, 1/54, 1/216 */
    v->d = 3;
    v->q = 27;
    for (i = 0; i < 27; ++i) {
      for (a = 0; a < 3; ++a) v->c[i][a] = ORC_D3Q27_C[i][a];
      v->w[i] = (i == 0) ? 8.0 / 27.0
                         : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
  } else if (lattice == 3) { /* D1Q3: one-dimensional stencil, textbook 2/3, 1/6 */
    v->d = 1;
    v->q = 3;
    for (i = 0; i < 3; ++i) {
      for (a = 0; a < 3; ++a) v->c[i][a] = ORC_D1Q3_C[i][a];
      v->w[i] = (i == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
    }
  } else {
    return -1;
  }
  for (i = 0; i < v->q; ++i) {
    int j, found = -1;
    for (j = 0; j < v->q; ++j)
      if (v->c[j][0] == -v->c[i][0] && v->c[j][1] == -v->c[i][1] &&
          v->c[j][2] == -v->c[i][2])
        found = j;
    v->opp[i] = found;
  }
  return 0;
}

/* Quadrature weights of Table "weights": (varpi_0, varpi_{i!=0}) for d=1,2,3;
   d = -1: the pointwise phi(x) (R8). */
static int orc_quad_weights(int quad_dim, double *w0, double *w1) {
  if (quad_dim == -1) { *w0 = 1.0; *w1 = 0.0; return 0; }
  if (quad_dim == 1) { *w0 = 1.0 / 2.0; *w1 = 1.0 / 4.0; return 0; }
  if (quad_dim == 2) { *w0 = 1.0 / 3.0; *w1 = 1.0 / 6.0; return 0; }
  if (quad_dim == 3) { *w0 = 1.0 / 6.0; *w1 = 5.0 / 36.0; return 0; }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Problem description shared by all entry points (passed from Python).      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int lattice;              /* 0 D2Q9, 1 D3Q19, 2 D3Q27 */
  int nx, ny, nz;           /* nz = 1 for D2Q9 */
  double tau;               /* BGK relaxation time, eq. (lbe) */
  double rho0;              /* reference density of the pressure datum (R2) */
  int quad_dim;             /* Table "weights" row: 1, 2 or 3 */
  unsigned quad_axes;       /* bit a: axis a enters eq. (quad) (R3) */
  unsigned walls;           /* bit a: solid first/last layer on axis a (R6) */
  const double *eps_ref;    /* phi at n_eps, N values, x fastest */
  const double *deps_dt;    /* d_t phi, N values, or NULL (static phi) */
  long long n_eps;
  double g[3];              /* uniform external force density (R5) */
  const double *force;      /* optional field, 3*N component-major, or NULL */
  const double *dforce_dt;  /* its time derivative, or NULL */
  long long n_force;
  int drag_model;           /* R9: 0 none, 1 Ergun-type drag */
  double drag_c1, drag_c2;  /* R9: viscous and inertial coefficients */
  double drag_d;            /* R9: particle diameter (lattice units) */
  double les_cs;            /* R10: Smagorinsky constant, 0 = plain BGK */
} orc_problem;

static size_t orc_ncells(const orc_problem *P) {
  return (size_t)P->nx * (size_t)P->ny * (size_t)P->nz;
}

static size_t orc_index(const orc_problem *P, int x, int y, int z) {
  return ((size_t)z * (size_t)P->ny + (size_t)y) * (size_t)P->nx + (size_t)x;
}

static int orc_wrap(int v, int n) {
  if (v < 0) return v + n;
  if (v >= n) return v - n;
  return v;
}

/* Cell (x,y,z) is solid when it lies in a wall layer (R6). */
static int orc_is_solid(const orc_problem *P, int x, int y, int z) {
  if ((P->walls & 1u) && (x == 0 || x == P->nx - 1)) return 1;
  if ((P->walls & 2u) && (y == 0 || y == P->ny - 1)) return 1;
  if ((P->walls & 4u) && (z == 0 || z == P->nz - 1)) return 1;
  return 0;
}

/* phi at time n at cell (x,y,z) with periodic wrap (R4). */
static double orc_eps_at(const orc_problem *P, long long n, int x, int y, int z) {
  size_t k = orc_index(P, orc_wrap(x, P->nx), orc_wrap(y, P->ny), orc_wrap(z, P->nz));
  if (P->deps_dt) {
    double dn = (double)(n - P->n_eps);
    return P->eps_ref[k] + dn * P->deps_dt[k];
  }
  return P->eps_ref[k];
}

static int orc_validate(const orc_problem *P, orc_vset *v) {
  if (orc_make_vset(P->lattice, v)) return -1;
  if (P->nx < 1 || P->ny < 1 || P->nz < 1) return -1;
  if (v->d == 2 && P->nz != 1) return -1;
  if (v->d == 1 && (P->ny != 1 || P->nz != 1)) return -1;
  if (!(P->tau > 0.5)) return -1;
  if (!P->eps_ref) return -1;
  {
    double w0, w1;
    if (orc_quad_weights(P->quad_dim, &w0, &w1)) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Macroscopic state of one cell at time n from its pre-collision           */
/* populations fc[0..Q-1] (Sec. 2.2, eqs. (density), (velocity),            */
/* (pressForce), (quad)).                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  double M0;     /* sum_i f_i */
  double J[3];   /* sum_i xi_i f_i */
  double I;      /* int_V phi dV by eq. (quad) */
  double rho;    /* rho~ = M0 / I, eq. (density) */
  double F[3];   /* total force sum_k F_k = F_ext + F_PC */
  double u[3];   /* eq. (velocity) */
} orc_macro;

static void orc_cell_macro(const orc_problem *P, const orc_vset *v, long long n,
                           int x, int y, int z, const double *fc, orc_macro *m) {
  int i, a;
  double w0, w1, e_c, e_p[3], e_m[3], nb, pc;
  size_t k = orc_index(P, x, y, z);

  /* zeroth and first moments of the populations */
  m->M0 = 0.0;
  for (i = 0; i < v->q; ++i) m->M0 = m->M0 + fc[i];
  for (a = 0; a < 3; ++a) {
    m->J[a] = 0.0;
    for (i = 0; i < v->q; ++i) m->J[a] = m->J[a] + (double)v->c[i][a] * fc[i];
  }

  /* volume fraction at the cell and at its face neighbours on each axis */
  e_c = orc_eps_at(P, n, x, y, z);
  for (a = 0; a < 3; ++a) {
    int dx = (a == 0), dy = (a == 1), dz = (a == 2);
    if (a < v->d) {
      e_p[a] = orc_eps_at(P, n, x + dx, y + dy, z + dz);
      e_m[a] = orc_eps_at(P, n, x - dx, y - dy, z - dz);
    } else {
      e_p[a] = e_c;
      e_m[a] = e_c;
    }
  }

  /* eq. (quad): int phi dV = varpi_0 phi(x) + varpi_1 sum of face neighbours
     phi(x - xi_k) over the quadrature axes (no diagonals) */
  orc_quad_weights(P->quad_dim, &w0, &w1);
  nb = 0.0;
  for (a = 0; a < 3; ++a) {
    if (P->quad_axes & (1u << a)) {
      nb = nb + e_p[a];
      nb = nb + e_m[a];
    }
  }
  m->I = w0 * e_c + w1 * nb;

  /* eq. (density) */
  m->rho = m->M0 / m->I;

  /* eq. (pressForce): F_PC = rho~ c_s^2 grad(phi), central differences */
  pc = m->rho / 3.0;
  for (a = 0; a < 3; ++a) {
    double grad = 0.5 * (e_p[a] - e_m[a]);
    double fext = P->g[a];
    if (P->force) {
      double fa = P->force[(size_t)a * orc_ncells(P) + k];
      if (P->dforce_dt) {
        double dn = (double)(n - P->n_force);
        fa = fa + dn * P->dforce_dt[(size_t)a * orc_ncells(P) + k];
      }
      fext = fext + fa;
    }
    m->F[a] = (a < v->d) ? fext + pc * grad : 0.0;
  }

  /* eq. (velocity): u = (sum xi f + dt/2 sum F) / sum f */
  if (!P->drag_model) {
    for (a = 0; a < 3; ++a) m->u[a] = (m->J[a] + 0.5 * m->F[a]) / m->M0;
    return;
  }

  /* R9: the phase-interaction drag F_D = -(b_lin + b_q |u|) u joins the
     force sum, taken implicitly in eq. (velocity): with b = J + F/2 (every
     other force) the velocity solves (M0 + (b_lin + b_q |u|)/2) u = b, so
     |u| = s is the positive root of (b_q/2) s^2 + (M0 + b_lin/2) s - |b| = 0,
     written without cancellation as s = 2|b| / (A + sqrt(A^2 + 2 b_q |b|)),
     A = M0 + b_lin/2.  Then u = b / (A + b_q s/2) and F += F_D, so that
     eq. (velocity) holds with the full force sum. */
  {
    double b[3], bn, e_x, one_m, nu, blin, bq, A, sp, den, fd;
    e_x = e_c;
    one_m = 1.0 - e_x;
    nu = (P->tau - 0.5) / 3.0;
    blin = m->rho * P->drag_c1 * one_m * one_m * nu / (e_x * P->drag_d * P->drag_d);
    bq = m->rho * P->drag_c2 * one_m / P->drag_d;
    bn = 0.0;
    for (a = 0; a < 3; ++a) {
      b[a] = m->J[a] + 0.5 * m->F[a];
      bn = bn + b[a] * b[a];
    }
    bn = sqrt(bn);
    A = m->M0 + 0.5 * blin;
    sp = 2.0 * bn / (A + sqrt(A * A + 2.0 * bq * bn));
    den = A + 0.5 * bq * sp;
    for (a = 0; a < 3; ++a) {
      m->u[a] = b[a] / den;
      fd = (blin + bq * sp) * m->u[a];
      m->F[a] = (a < v->d) ? m->F[a] - fd : 0.0;
    }
  }
}

/* eq. (feq) with the zeroth moment M0 in place of rho~ phi:
   f_i^eq = w_i M0 (1 + xi.u/c_s^2 + (xi xi - c_s^2 I):uu/(2 c_s^4)). */
static double orc_feq(const orc_vset *v, int i, double M0, const double *u, double usq) {
  double cu = 0.0;
  int a;
  for (a = 0; a < 3; ++a) cu = cu + (double)v->c[i][a] * u[a];
  return v->w[i] * M0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

/* Guo forcing term of Sec. 2.2,
   Omega_i^F = (1 - 1/(2 tau)) w_i [xi_a/c_s^2 + (xi_a xi_b - c_s^2 d_ab) u_b / c_s^4] F_a,
   with 1/c_s^2 = 3 and 1/c_s^4 = 9 this is
   (1 - 1/(2 tau)) w_i (3 (xi.F - u.F) + 9 (xi.u)(xi.F)). */
static double orc_guo(const orc_vset *v, int i, double cf, const double *u,
                      const double *F, double uF) {
  double cu = 0.0, cF = 0.0;
  int a;
  for (a = 0; a < 3; ++a) cu = cu + (double)v->c[i][a] * u[a];
  for (a = 0; a < 3; ++a) cF = cF + (double)v->c[i][a] * F[a];
  return cf * v->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
}

/* ------------------------------------------------------------------------ */
/* Public entry points (ctypes).  All return 0 on success, -1 on bad input.  */
/* ------------------------------------------------------------------------ */

static int orc_threads = 0;

void oracle_set_threads(int n) { orc_threads = n; }

int oracle_q(int lattice) {
  orc_vset v;
  if (orc_make_vset(lattice, &v)) return -1;
  return v.q;
}

/* Copy the velocity set out (for pinning tests): c[Q*3] ints, w[Q], opp[Q]. */
int oracle_velocity_set(int lattice, int *c, double *w, int *opp) {
  orc_vset v;
  int i, a;
  if (orc_make_vset(lattice, &v)) return -1;
  for (i = 0; i < v.q; ++i) {
    for (a = 0; a < 3; ++a) c[i * 3 + a] = v.c[i][a];
    w[i] = v.w[i];
    opp[i] = v.opp[i];
  }
  return v.q;
}

int oracle_quad_weights(int quad_dim, double *w) {
  return orc_quad_weights(quad_dim, &w[0], &w[1]);
}

/* Equilibrium and forcing of one cell, for moment pins: feq[Q], omega_f[Q]. */
int oracle_cell_terms(int lattice, double M0, const double *u, const double *F, double tau,
                      double *feq, double *omega_f) {
  orc_vset v;
  int i;
  double usq, uF, cf;
  if (orc_make_vset(lattice, &v)) return -1;
  usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  cf = 1.0 - 0.5 / tau;
  for (i = 0; i < v.q; ++i) {
    feq[i] = orc_feq(&v, i, M0, u, usq);
    omega_f[i] = orc_guo(&v, i, cf, u, F, uF);
  }
  return 0;
}

/* Initial populations (eq. (equilibrium)): f_i = w_i rho~0 phi poly_i(u0) with
   rho~0 = rho0 + p0 / c_s^2.  Bits of `mode`:
     1  use int phi dV (eq. (feq)) instead of phi as the mass factor;
     2  shift the equilibrium velocity by the Guo half force, u_eq = u0 -
        F / (2 M0), with F the force sum of time n evaluated on these
        populations, so that eq. (velocity) returns u0 at time n.
   p0, u0 may be NULL (rest state).  Solid cells get 0. */
int oracle_init(const orc_problem *P, const double *p0, const double *u0,
                int mode, long long n, double *f) {
  orc_vset v;
  int x, y, z, i, a;
  size_t N;
  if (orc_validate(P, &v)) return -1;
  N = orc_ncells(P);
  for (z = 0; z < P->nz; ++z)
    for (y = 0; y < P->ny; ++y)
      for (x = 0; x < P->nx; ++x) {
        size_t k = orc_index(P, x, y, z);
        double u[3] = {0.0, 0.0, 0.0}, usq, rt, mass;
        if (orc_is_solid(P, x, y, z)) {
          for (i = 0; i < v.q; ++i) f[k * v.q + i] = 0.0;
          continue;
        }
        if (u0)
          for (a = 0; a < v.d; ++a) u[a] = u0[(size_t)a * N + k];
        usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        rt = P->rho0 + (p0 ? 3.0 * p0[k] : 0.0);
        if (mode & 1) {
          double w0, w1, nb = 0.0;
          orc_quad_weights(P->quad_dim, &w0, &w1);
          for (a = 0; a < 3; ++a) {
            if (P->quad_axes & (1u << a)) {
              int dx = (a == 0), dy = (a == 1), dz = (a == 2);
              nb = nb + orc_eps_at(P, n, x + dx, y + dy, z + dz);
              nb = nb + orc_eps_at(P, n, x - dx, y - dy, z - dz);
            }
          }
          mass = rt * (w0 * orc_eps_at(P, n, x, y, z) + w1 * nb);
        } else {
          mass = rt * orc_eps_at(P, n, x, y, z);
        }
        for (i = 0; i < v.q; ++i) f[k * v.q + i] = orc_feq(&v, i, mass, u, usq);
        if (mode & 2) {
          orc_macro m;
          orc_cell_macro(P, &v, n, x, y, z, f + k * v.q, &m);
          for (a = 0; a < 3; ++a) u[a] = u[a] - 0.5 * m.F[a] / m.M0;
          usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
          for (i = 0; i < v.q; ++i) f[k * v.q + i] = orc_feq(&v, i, mass, u, usq);
        }
      }
  return 0;
}

/* One time step n -> n+1 (eq. (lbe)): collide every fluid cell with the
   macroscopic state of time n, then push to x + xi_i (periodic), or bounce
   back to x as the opposite direction when x + xi_i is solid (R6). */
int oracle_step(const orc_problem *P, long long n, const double *f, double *fnew) {
  orc_vset v;
  size_t N;
  double omega, cf;
  long row;
  if (orc_validate(P, &v)) return -1;
  N = orc_ncells(P);
  omega = 1.0 / P->tau;
  cf = 1.0 - 0.5 / P->tau;
  memset(fnew, 0, N * (size_t)v.q * sizeof(double));
  /* rows (y,z) are independent: each writes only its own cells' slots and
     the slots its populations stream into, which no other cell writes */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(orc_threads > 0 ? orc_threads : omp_get_max_threads())
#endif
  for (row = 0; row < (long)P->ny * P->nz; ++row) {
    int x, i;
    int y = (int)(row % P->ny), z = (int)(row / P->ny);
    for (x = 0; x < P->nx; ++x) {
        size_t k = orc_index(P, x, y, z);
        const double *fc = f + k * v.q;
        orc_macro m;
        double usq, uF;
        if (orc_is_solid(P, x, y, z)) continue;
        double om = omega, cfl = cf;
        orc_cell_macro(P, &v, n, x, y, z, fc, &m);
        usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
        uF = m.u[0] * m.F[0] + m.u[1] * m.F[1] + m.u[2] * m.F[2];
        if (P->les_cs > 0.0) {
          /* R10: Pi^neq_ab = sum_i xi_ia xi_ib (f_i - f_i^eq), Q = |Pi^neq| */
          double pi[3][3], Q2 = 0.0, teff;
          int a, b;
          for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) pi[a][b] = 0.0;
          for (i = 0; i < v.q; ++i) {
            double fneq = fc[i] - orc_feq(&v, i, m.M0, m.u, usq);
            for (a = 0; a < 3; ++a)
              for (b = 0; b < 3; ++b)
                pi[a][b] = pi[a][b] + (double)v.c[i][a] * (double)v.c[i][b] * fneq;
          }
          for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) Q2 = Q2 + pi[a][b] * pi[a][b];
          teff = 0.5 * (P->tau + sqrt(P->tau * P->tau +
                                      18.0 * sqrt(2.0) * P->les_cs * P->les_cs * sqrt(Q2) / m.M0));
          om = 1.0 / teff;
          cfl = 1.0 - 0.5 / teff;
        }
        for (i = 0; i < v.q; ++i) {
          double feq = orc_feq(&v, i, m.M0, m.u, usq);
          double S = orc_guo(&v, i, cfl, m.u, m.F, uF);
          double fstar = fc[i] + om * (feq - fc[i]) + S;
          int xn = orc_wrap(x + v.c[i][0], P->nx);
          int yn = orc_wrap(y + v.c[i][1], P->ny);
          int zn = orc_wrap(z + v.c[i][2], P->nz);
          /* a wall layer is the first/last layer, so a step that would
             leave the array through a wall axis always lands in a solid cell */
          if (orc_is_solid(P, xn, yn, zn))
            fnew[k * v.q + v.opp[i]] = fstar;
          else
            fnew[orc_index(P, xn, yn, zn) * v.q + i] = fstar;
      }
    }
  }
  return 0;
}

/* nsteps steps starting at time n0; result is left in f (work is scratch of
   the same size). */
int oracle_run(const orc_problem *P, long long n0, long long nsteps, double *f, double *work) {
  orc_vset v;
  long long s;
  size_t bytes;
  if (orc_validate(P, &v)) return -1;
  bytes = orc_ncells(P) * (size_t)v.q * sizeof(double);
  for (s = 0; s < nsteps; ++s) {
    if (oracle_step(P, n0 + s, f, work)) return -1;
    memcpy(f, work, bytes);
  }
  return 0;
}

/* nsteps steps starting at time n0 with per-step fields: before step s the
   volume fraction is eps_series[s*N..] (and the force field
   force_series[s*3N..] when given), both exact at time n0+s; the problem's
   own phi and field pointers are replaced for the duration of the call. */
int oracle_run_series(const orc_problem *P, long long n0, long long nsteps,
                      const double *eps_series, const double *force_series,
                      double *f, double *work) {
  orc_vset v;
  orc_problem Q;
  long long s;
  size_t N, bytes;
  if (orc_validate(P, &v)) return -1;
  N = orc_ncells(P);
  bytes = N * (size_t)v.q * sizeof(double);
  Q = *P;
  Q.deps_dt = NULL;
  Q.dforce_dt = NULL;
  for (s = 0; s < nsteps; ++s) {
    if (eps_series) Q.eps_ref = eps_series + (size_t)s * N;
    if (force_series) Q.force = force_series + (size_t)s * 3 * N;
    if (oracle_step(&Q, n0 + s, f, work)) return -1;
    memcpy(f, work, bytes);
  }
  return 0;
}

/* Macroscopic fields at time n from pre-collision populations f:
   rho~ (eq. (density)), p = c_s^2 (rho~ - rho0) (R2), u (eq. (velocity)),
   and the zeroth moment M0.  Any output pointer may be NULL.  Solid cells
   report zeros. */
int oracle_moments(const orc_problem *P, long long n, const double *f, double *rho,
                   double *p, double *u, double *M0) {
  orc_vset v;
  size_t N;
  int x, y, z, a;
  if (orc_validate(P, &v)) return -1;
  N = orc_ncells(P);
  for (z = 0; z < P->nz; ++z)
    for (y = 0; y < P->ny; ++y)
      for (x = 0; x < P->nx; ++x) {
        size_t k = orc_index(P, x, y, z);
        orc_macro m;
        if (orc_is_solid(P, x, y, z)) {
          if (rho) rho[k] = 0.0;
          if (p) p[k] = 0.0;
          if (M0) M0[k] = 0.0;
          if (u)
            for (a = 0; a < 3; ++a) u[(size_t)a * N + k] = 0.0;
          continue;
        }
        orc_cell_macro(P, &v, n, x, y, z, f + k * v.q, &m);
        if (rho) rho[k] = m.rho;
        if (p) p[k] = (m.rho - P->rho0) / 3.0;
        if (M0) M0[k] = m.M0;
        if (u)
          for (a = 0; a < 3; ++a) u[(size_t)a * N + k] = m.u[a];
      }
  return 0;
}

/* Total force sum_k F_k per cell at time n (3*N component-major): used by
   the momentum-balance pin. */
int oracle_forces(const orc_problem *P, long long n, const double *f, double *F) {
  orc_vset v;
  size_t N;
  int x, y, z, a;
  if (orc_validate(P, &v)) return -1;
  N = orc_ncells(P);
  for (z = 0; z < P->nz; ++z)
    for (y = 0; y < P->ny; ++y)
      for (x = 0; x < P->nx; ++x) {
        size_t k = orc_index(P, x, y, z);
        orc_macro m;
        if (orc_is_solid(P, x, y, z)) {
          for (a = 0; a < 3; ++a) F[(size_t)a * N + k] = 0.0;
          continue;
        }
        orc_cell_macro(P, &v, n, x, y, z, f + k * v.q, &m);
        for (a = 0; a < 3; ++a) F[(size_t)a * N + k] = m.F[a];
      }
  return 0;
}

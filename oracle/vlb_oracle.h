/*
 * vlb_oracle.h -- plain FP64 CPU oracle for the volumetric lattice Boltzmann
 * method on a curvilinear mesh (H. Chen, "Volumetric Lattice Boltzmann Models
 * in General Curvilinear Coordinates: Theoretical Formulation", section 2).
 *
 * TEST INFRASTRUCTURE.  This library exists to check the CUDA path.  Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg
 * load it; the product library never does, and the two share no source.
 *
 * Everything is computed literally, cell by cell and direction by direction,
 * in double precision, in the order the paper states the equations:
 *   geometry     : D_{+-i} (Eq. 1), g_i and beta_i (Eq. 3), g_ij (Eq. 4),
 *                  J (Eq. 5), g^i (Eq. 7), g^ij (Eq. 8),
 *                  Theta^i_j(q + c_a, q) (Eq. 11)
 *   one time step: f = N/J (Eq. 14), rho and U (Eqs. 15, 17), the BGK
 *                  collision (Eq. 20 with M = -delta/tau), the equilibrium
 *                  (Eq. 33) with U~ = U + F/(2 rho) (text after Eq. 32),
 *                  deltaPi (Eq. 30), deltaN (Eq. 31), the inertial force
 *                  J F^i (Eq. 27), N' = N + Omega + deltaN (Eq. 12) and the
 *                  one-to-one advection N(q + c_a, t + 1) = N'(q, t) (Eq. 22)
 *   output       : rho and u = U^i g_i (Eq. 34)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the implicit relation between F and N' (text after Eq. 31) is solved
 *     by fixed-point iteration from F = 0 until max|dF| <= tol*max(rho,|F|);
 *     the returned N' is evaluated with the final F;
 *   - walls are index-space halfway bounce-back; ghost nodes behind a wall
 *     are linear extrapolations; on links that cross a wall Theta is either
 *     zero (wall_links = 0: the reflected particle never travels the link) or
 *     taken from the ghost nodes (wall_links = 1);
 *     a moving wall subtracts J rho (f^eq_a - f^eq_abar) evaluated with the
 *     paper's equilibrium at rho = 1, U = U~ = U_wall;
 *   - an external body force G adds rho G.g^i to F^i inside the fixed point;
 *   - velocity sets: D3Q19 as listed in section 2.1 and its 2D restriction
 *     D2Q9, with the standard weights (the paper states none); T0 = 1/3.
 *     D3Q39 (speeds up to 3; T0 = 2/3), a set that meets the isotropy
 *     conditions of Eq. 10 to 6th order as the paper asks, so that the third
 *     moment Q^eq of the equilibrium is matched exactly; periodic meshes
 *     (every axis at least 3 cells) only.
 *
 * Parity pins: the test suite checks this library against closed forms,
 * moment identities, conservation laws, a textbook Cartesian LBM on the
 * identity map and the Couette solution; nothing here is "parity unpinned"
 * except the long-time dynamics on an arbitrary curved mesh, for which the
 * paper prints no values.
 */
#ifndef VLB_ORACLE_H
#define VLB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VLBO_OK 0
#define VLBO_EINVAL 1
#define VLBO_EGEOM 2
#define VLBO_ENOCONV 3
#define VLBO_ENOMEM 4

#define VLBO_PERIODIC 0
#define VLBO_WALL 1

#define VLBO_QMAX 39

/* A structured mesh: node positions x(q) on the index lattice q (section 2.1).
 * x is C-ordered [n0][n1][n2][dim] (n2 = 1 when dim = 2) and is only borrowed
 * by vlbo_cell_geometry; vlbo_create copies it. */
typedef struct {
  int32_t dim;             /* 2 or 3 */
  int32_t q;               /* 9 (D2Q9, dim 2), 19 (D3Q19, dim 3) or 39 (D3Q39, dim 3) */
  int64_t n[3];
  const double *x;
  int32_t bc[3];           /* VLBO_PERIODIC or VLBO_WALL per axis */
  double shift[3][3];      /* periodic image across the +end of axis a: R_a x + shift[a] */
  double rot[3][9];        /* R_a row-major; an all-zero matrix means identity */
  double dx;               /* representative spacing Delta x of Eq. 3; 0 means 1 */
  int32_t wall_links;      /* Theta on links that cross a wall: 0 zero (the link reflects
                              in place), 1 from the linearly extrapolated ghost nodes */
} vlbo_mesh;

typedef struct {
  double tau;
  double body_force[3];         /* Euclidean acceleration G */
  double wall_u[3][2][3];       /* wall on axis a, side s (0: index 0, 1: index n-1): translation */
  double wall_omega[3][2][3];   /* and angular velocity about the origin */
  int32_t max_iter;             /* fixed-point cap; 0 means 200 */
  double tol;                   /* fixed-point tolerance; 0 means 1e-14 */
} vlbo_params;

/* Geometry of one cell (section 2.1) plus the per-link data the step needs. */
typedef struct {
  double J;
  double g_low[3][3];             /* g_i, row i (Eq. 3) */
  double g_up[3][3];              /* g^i, row i (Eq. 7) */
  double gij[3][3];               /* g_ij (Eq. 4) */
  double ginv[3][3];              /* g^ij (Eq. 8) */
  double theta[VLBO_QMAX][3][3];  /* Theta^i_j(q + c_a, q) as [a][i][j] (Eq. 11) */
  int32_t wall_link[VLBO_QMAX];   /* 1 when q + c_a lies beyond a wall */
  double uw[VLBO_QMAX][3];        /* U_wall^i = u_wall . g^i for wall links */
  double G[3];                    /* G^i = G . g^i */
} vlbo_cell;

typedef struct vlbo_sim vlbo_sim;

/* Velocity set: c[a][3] (unused components zero), weights w[a], T0. */
int vlbo_lattice(int32_t q, int32_t *c, double *w, double *T0);

/* Position of any index p, including ghost and periodic-image nodes. */
int vlbo_position(const vlbo_mesh *m, const int64_t p[3], double out[3]);

/* Geometry of in-domain cell qi; params may be NULL (no wall motion, G = 0). */
int vlbo_cell_geometry(const vlbo_mesh *m, const vlbo_params *p, const int64_t qi[3],
                       vlbo_cell *out);

/* Eq. 33 for one cell: ginv is g^ij row-major 3x3. */
int vlbo_equilibrium(int32_t q, double rho, const double U[3], const double Ut[3],
                     const double ginv[9], double *feq);

/* One collision (Eqs. 12, 20, 27, 30, 31, 33) of the arrived populations N.
 * Outputs (any may be NULL): N' (Np), F^i, f^eq, deltaPi (3x3), deltaN, Omega,
 * and the fixed-point iteration count. */
int vlbo_collide(int32_t q, const vlbo_cell *cell, const vlbo_params *p, const double *N,
                 double *Np, double *F, double *feq, double *dPi, double *dN,
                 double *Om, int32_t *iters);

/* Whole-mesh simulation with two population arrays (collide, then stream). */
int vlbo_create(const vlbo_mesh *m, const vlbo_params *p, vlbo_sim **out);
void vlbo_destroy(vlbo_sim *s);
/* N_a = J f^eq_a(rho, U, U~ = U) with U^i = u . g^i; rho [ncell], u [ncell][dim]. */
int vlbo_init(vlbo_sim *s, const double *rho, const double *u);
/* nsteps time steps; the cells of a step may run on several threads
 * (OpenMP), with the same result bit for bit as on one. */
int vlbo_step(vlbo_sim *s, int64_t nsteps);
/* Threads vlbo_step may use from now on in this process (n <= 0 leaves the
 * setting); returns the count in effect (1 without OpenMP). */
int vlbo_set_threads(int32_t n);
/* rho [ncell], u and u_tilde [ncell][dim] (Euclidean, Eq. 34 with U and U~),
 * F [ncell][dim] index components, totals[7] = mass, P (3), M (3). */
int vlbo_moments(vlbo_sim *s, double *rho, double *u, double *u_tilde, double *F,
                 double *totals);
int vlbo_get_state(const vlbo_sim *s, double *N);   /* [q][ncell], arrived populations */
int vlbo_set_state(vlbo_sim *s, const double *N);
int vlbo_get_cell(const vlbo_sim *s, int64_t idx, vlbo_cell *out);
/* Largest fixed-point iteration count seen by the last step or moments call. */
int32_t vlbo_last_iters(const vlbo_sim *s);

#ifdef __cplusplus
}
#endif
#endif

/*
 * vlb_oracle.c -- plain FP64 CPU oracle for the volumetric curvilinear lattice
 * Boltzmann method (H. Chen, section 2).  TEST INFRASTRUCTURE: see
 * vlb_oracle.h for what may use it and for the readings it takes.
 *
 * Built with -O2 -ffp-contract=off so that every product and sum is rounded
 * the way it is written.  No blocking, fusion or reordering: each function
 * evaluates one equation of the paper, in its notation, with explicit loops.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "vlb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Velocity sets (section 2.1).  D3Q19 in the order the paper lists it; D2Q9 is
 * its restriction to the plane.  Weights are the standard ones that satisfy
 * the isotropy conditions of Eq. 10 up to 4th order with T0 = 1/3. */

static const int32_t C9[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int32_t C19[19][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                               1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* D3Q39: a velocity set with moment isotropy to 6th order (Eq. 10 in full),
 * T0 = 2/3: the rest vector, the 6 unit axis vectors, the 8 corner vectors
 * (+-1, +-1, +-1), 6 axis vectors of length 2, the 12 vectors (+-2, +-2, 0) and
 * permutations, and 6 axis vectors of length 3; weights 1/12, 1/12, 1/27,
 * 2/135, 1/432 and 1/1620 (a set from the literature on higher-order lattice
 * Boltzmann models; the tests check Eq. 10 on it to 6th order exactly). */
static int32_t C39[39][3];
static double W39[39];
static int c39_ready = 0;
static void c39_fill(void) {
  int k = 0;
  C39[k][0] = C39[k][1] = C39[k][2] = 0;
  W39[k++] = 1.0 / 12.0;
  for (int d = 0; d < 3; d++)
    for (int s = 1; s >= -1; s -= 2) {
      C39[k][0] = C39[k][1] = C39[k][2] = 0;
      C39[k][d] = s;
      W39[k++] = 1.0 / 12.0;
    }
  for (int x = 1; x >= -1; x -= 2)
    for (int y = 1; y >= -1; y -= 2)
      for (int z = 1; z >= -1; z -= 2) {
        C39[k][0] = x;
        C39[k][1] = y;
        C39[k][2] = z;
        W39[k++] = 1.0 / 27.0;
      }
  for (int d = 0; d < 3; d++)
    for (int s = 2; s >= -2; s -= 4) {
      C39[k][0] = C39[k][1] = C39[k][2] = 0;
      C39[k][d] = s;
      W39[k++] = 2.0 / 135.0;
    }
  for (int d = 0; d < 3; d++)
    for (int e = d + 1; e < 3; e++)
      for (int s = 2; s >= -2; s -= 4)
        for (int t = 2; t >= -2; t -= 4) {
          C39[k][0] = C39[k][1] = C39[k][2] = 0;
          C39[k][d] = s;
          C39[k][e] = t;
          W39[k++] = 1.0 / 432.0;
        }
  for (int d = 0; d < 3; d++)
    for (int s = 3; s >= -3; s -= 6) {
      C39[k][0] = C39[k][1] = C39[k][2] = 0;
      C39[k][d] = s;
      W39[k++] = 1.0 / 1620.0;
    }
  c39_ready = 1;
}

static const int32_t (*lat_c(int32_t q))[3] {
  if (q == 39 && !c39_ready) c39_fill();
  return q == 9 ? C9 : q == 19 ? C19 : (const int32_t(*)[3])C39;
}
static const double *lat_w(int32_t q) {
  if (q == 39 && !c39_ready) c39_fill();
  return q == 9 ? W9 : q == 19 ? W19 : W39;
}
static int lat_dim(int32_t q) { return q == 9 ? 2 : 3; }
/* the lattice constant T0 of Eq. 10 */
static double lat_T0(int32_t q) { return q == 39 ? 2.0 / 3.0 : 1.0 / 3.0; }
static int lat_known(int32_t q) { return q == 9 || q == 19 || q == 39; }

/* index of the opposite direction c_abar = -c_a, found by search once */
static int OPP9[9], OPP19[19], OPP39[39], opp_ready = 0;
static void opp_fill(void) {
  for (int t = 0; t < 3; t++) {
    int32_t q = t == 0 ? 9 : t == 1 ? 19 : 39;
    const int32_t(*c)[3] = lat_c(q);
    int *o = t == 0 ? OPP9 : t == 1 ? OPP19 : OPP39;
    for (int a = 0; a < q; a++)
      for (int b = 0; b < q; b++)
        if (c[b][0] == -c[a][0] && c[b][1] == -c[a][1] && c[b][2] == -c[a][2]) o[a] = b;
  }
  opp_ready = 1;
}
static int opposite(int32_t q, int a) {
  if (!opp_ready) opp_fill();
  return q == 9 ? OPP9[a] : q == 19 ? OPP19[a] : OPP39[a];
}

static double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

int vlbo_lattice(int32_t q, int32_t *c, double *w, double *t0) {
  if (!lat_known(q)) return VLBO_EINVAL;
  const int32_t(*cc)[3] = lat_c(q);
  const double *ww = lat_w(q);
  for (int a = 0; a < q; a++) {
    if (c)
      for (int d = 0; d < 3; d++) c[3 * a + d] = cc[a][d];
    if (w) w[a] = ww[a];
  }
  if (t0) *t0 = lat_T0(q);
  return VLBO_OK;
}

/* ------------------------------------------------------------------------- */
/* Mesh positions, including ghosts (section 2.1 defines D_{+-i} from the
 * neighbouring vertices; off the mesh the neighbours come from the periodic
 * image or, behind a wall, from linear extrapolation). */

static int64_t node_index(const vlbo_mesh *m, const int64_t p[3]) {
  return (p[0] * m->n[1] + p[1]) * m->n[2] + p[2];
}

static int rot_is_zero(const double *r) {
  for (int k = 0; k < 9; k++)
    if (r[k] != 0.0) return 0;
  return 1;
}

/* y = R x (forward) or y = R^T x (backward); identity when R is all zero */
static void apply_rot(const double *r, int dim, const double x[3], double y[3], int transpose) {
  if (rot_is_zero(r)) {
    for (int d = 0; d < 3; d++) y[d] = x[d];
    return;
  }
  for (int i = 0; i < 3; i++) {
    y[i] = 0.0;
    if (i >= dim) continue;
    for (int j = 0; j < dim; j++) y[i] += (transpose ? r[3 * j + i] : r[3 * i + j]) * x[j];
  }
}

int vlbo_position(const vlbo_mesh *m, const int64_t p[3], double out[3]) {
  int dim = m->dim;
  for (int a = 0; a < dim; a++) {
    if (p[a] >= 0 && p[a] < m->n[a]) continue;
    int64_t r[3] = {p[0], p[1], p[2]};
    double y[3], z[3];
    if (m->bc[a] == VLBO_PERIODIC) {
      if (p[a] >= m->n[a]) {
        r[a] = p[a] - m->n[a];
        vlbo_position(m, r, y);
        apply_rot(m->rot[a], dim, y, z, 0);
        for (int d = 0; d < 3; d++) out[d] = z[d] + (d < dim ? m->shift[a][d] : 0.0);
      } else {
        r[a] = p[a] + m->n[a];
        vlbo_position(m, r, y);
        for (int d = 0; d < 3; d++) y[d] -= (d < dim ? m->shift[a][d] : 0.0);
        apply_rot(m->rot[a], dim, y, out, 1);
      }
      return VLBO_OK;
    }
    /* wall: x(p) = 2 x(p -+ e_a) - x(p -+ 2 e_a), toward the inside */
    int64_t r2[3] = {p[0], p[1], p[2]};
    if (p[a] < 0) {
      r[a] = p[a] + 1;
      r2[a] = p[a] + 2;
    } else {
      r[a] = p[a] - 1;
      r2[a] = p[a] - 2;
    }
    vlbo_position(m, r, y);
    vlbo_position(m, r2, z);
    for (int d = 0; d < 3; d++) out[d] = 2.0 * y[d] - z[d];
    return VLBO_OK;
  }
  int64_t k = node_index(m, p);
  for (int d = 0; d < 3; d++) out[d] = d < dim ? m->x[k * dim + d] : 0.0;
  return VLBO_OK;
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Tangent basis g_i at any index p (Eqs. 1 and 3). */
static int tangents(const vlbo_mesh *m, const int64_t p[3], double gl[3][3]) {
  double dx = m->dx > 0.0 ? m->dx : 1.0;
  double x0[3];
  vlbo_position(m, p, x0);
  memset(gl, 0, 9 * sizeof(double));
  for (int i = 0; i < m->dim; i++) {
    int64_t pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
    pp[i] += 1;
    pm[i] -= 1;
    double xp[3], xm[3], Dp[3], Dm[3], diff[3];
    vlbo_position(m, pp, xp);
    vlbo_position(m, pm, xm);
    for (int d = 0; d < 3; d++) {
      Dp[d] = xp[d] - x0[d]; /* D_{+i}(q) = x(q_{+i}) - x(q) */
      Dm[d] = xm[d] - x0[d]; /* D_{-i}(q) = x(q_{-i}) - x(q) */
      diff[d] = Dp[d] - Dm[d];
    }
    double nd = norm3(diff);
    if (!(nd > 0.0)) return VLBO_EGEOM;
    double beta = (norm3(Dp) + norm3(Dm)) / nd;
    for (int d = 0; d < 3; d++) gl[i][d] = beta * diff[d] / (2.0 * dx);
  }
  return VLBO_OK;
}

/* J (Eq. 5) and the co-tangent basis g^i (Eq. 7). In 2D the third tangent is
 * the unit normal of the plane, so J = g_1 x g_2 . z. */
static int dual_basis(int dim, const double gl[3][3], double *J, double gu[3][3]) {
  memset(gu, 0, 9 * sizeof(double));
  if (dim == 2) {
    double j = gl[0][0] * gl[1][1] - gl[0][1] * gl[1][0];
    *J = j;
    if (!(j > 0.0)) return VLBO_EGEOM;
    gu[0][0] = gl[1][1] / j;
    gu[0][1] = -gl[1][0] / j;
    gu[1][0] = -gl[0][1] / j;
    gu[1][1] = gl[0][0] / j;
    return VLBO_OK;
  }
  double c12[3], c23[3], c31[3];
  cross3(gl[0], gl[1], c12);
  cross3(gl[1], gl[2], c23);
  cross3(gl[2], gl[0], c31);
  double j = dot3(c12, gl[2]);
  *J = j;
  if (!(j > 0.0)) return VLBO_EGEOM;
  for (int d = 0; d < 3; d++) {
    gu[0][d] = c23[d] / j;
    gu[1][d] = c31[d] / j;
    gu[2][d] = c12[d] / j;
  }
  return VLBO_OK;
}

int vlbo_cell_geometry(const vlbo_mesh *m, const vlbo_params *prm, const int64_t qi[3],
                       vlbo_cell *out) {
  int dim = m->dim, q = m->q;
  if ((dim == 2 && q != 9) || (dim == 3 && q != 19 && q != 39)) return VLBO_EINVAL;
  if (q == 39)
    for (int d = 0; d < dim; d++)
      if (m->bc[d] == VLBO_WALL) return VLBO_EINVAL; /* periodic meshes only */
  const int32_t(*c)[3] = lat_c(q);
  memset(out, 0, sizeof(*out));
  int rc = tangents(m, qi, out->g_low);
  if (rc) return rc;
  rc = dual_basis(dim, out->g_low, &out->J, out->g_up);
  if (rc) return rc;
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) {
      out->gij[i][j] = dot3(out->g_low[i], out->g_low[j]); /* Eq. 4 */
      out->ginv[i][j] = dot3(out->g_up[i], out->g_up[j]); /* Eq. 8 */
    }
  for (int i = 0; i < dim; i++)
    out->G[i] = prm ? dot3(prm->body_force, out->g_up[i]) : 0.0;

  for (int a = 1; a < q; a++) {
    int64_t p[3] = {qi[0] + c[a][0], qi[1] + c[a][1], qi[2] + c[a][2]};
    int wall_axis = -1, side = 0;
    for (int d = 0; d < dim; d++) {
      if (m->bc[d] != VLBO_WALL) continue;
      if (p[d] < 0 || p[d] >= m->n[d]) {
        wall_axis = d;
        side = p[d] < 0 ? 0 : 1;
        break;
      }
    }
    if (wall_axis >= 0) {
      /* bounce-back link; with wall_links = 0 it carries no curved-path
       * advection and Theta = 0 */
      out->wall_link[a] = 1;
      if (prm) {
        /* rigid wall motion evaluated at the wall point halfway to the ghost node */
        int64_t g[3] = {qi[0], qi[1], qi[2]};
        g[wall_axis] += side ? 1 : -1;
        double x0[3], xg[3], xw[3], uwv[3], om[3];
        vlbo_position(m, qi, x0);
        vlbo_position(m, g, xg);
        for (int d = 0; d < 3; d++) {
          xw[d] = 0.5 * (x0[d] + xg[d]);
          om[d] = prm->wall_omega[wall_axis][side][d];
        }
        cross3(om, xw, uwv);
        for (int d = 0; d < 3; d++) uwv[d] += prm->wall_u[wall_axis][side][d];
        for (int i = 0; i < dim; i++) out->uw[a][i] = dot3(uwv, out->g_up[i]);
      }
      if (m->wall_links != 1) continue;
      /* wall_links = 1: Theta from the tangents at the extrapolated ghost node */
    }
    double gp[3][3];
    rc = tangents(m, p, gp);
    if (rc) return rc;
    /* Theta^i_j(q + c_a, q) = [g_j(q + c_a) - g_j(q)] . g^i(q)   (Eq. 11) */
    for (int i = 0; i < dim; i++)
      for (int j = 0; j < dim; j++) {
        double dg[3];
        for (int d = 0; d < 3; d++) dg[d] = gp[j][d] - out->g_low[j][d];
        out->theta[a][i][j] = dot3(dg, out->g_up[i]);
      }
  }
  return VLBO_OK;
}

/* ------------------------------------------------------------------------- */
/* Equilibrium, Eq. 33.  The two bracketed tensors do not depend on the
 * direction, so they are formed once per call:
 *   B^ij  = (g^ij - delta^ij) T0 + U~^i U~^j
 *   C^ijk = T0 [(g^ij U~^k - delta^ij U^k) + (g^jk U~^i - delta^jk U^i)
 *               + (g^ki U~^j - delta^ki U^j)] + U~^i U~^j U~^k
 * and each direction contracts them with its Hermite tensors. */
int vlbo_equilibrium(int32_t q, double rho, const double U[3], const double Ut[3],
                     const double ginv[9], double *feq) {
  if (!lat_known(q)) return VLBO_EINVAL;
  const double T0 = lat_T0(q);
  int D = lat_dim(q);
  const int32_t(*c)[3] = lat_c(q);
  const double *w = lat_w(q);
  double B[3][3], C[3][3][3];
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) B[i][j] = (ginv[3 * i + j] - kd(i, j)) * T0 + Ut[i] * Ut[j];
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++)
      for (int k = 0; k < D; k++)
        C[i][j][k] = T0 * ((ginv[3 * i + j] * Ut[k] - kd(i, j) * U[k]) +
                           (ginv[3 * j + k] * Ut[i] - kd(j, k) * U[i]) +
                           (ginv[3 * k + i] * Ut[j] - kd(k, i) * U[j])) +
                     Ut[i] * Ut[j] * Ut[k];
  for (int a = 0; a < q; a++) {
    double s = 1.0;
    for (int i = 0; i < D; i++) s += c[a][i] * U[i] / T0;
    for (int i = 0; i < D; i++)
      for (int j = 0; j < D; j++) {
        double h2 = c[a][i] * c[a][j] / T0 - kd(i, j);
        s += h2 * B[i][j] / (2.0 * T0);
      }
    for (int i = 0; i < D; i++)
      for (int j = 0; j < D; j++)
        for (int k = 0; k < D; k++) {
          double h3 = c[a][i] * c[a][j] * c[a][k] -
                      T0 * (c[a][i] * kd(j, k) + c[a][j] * kd(k, i) + c[a][k] * kd(i, j));
          s += h3 * C[i][j][k] / (6.0 * T0 * T0 * T0);
        }
    feq[a] = rho * w[a] * s;
  }
  return VLBO_OK;
}

/* One evaluation of the collision for a given inertial force F.
 * Returns the updated force in Fnew (J F^i of Eq. 27 divided by J, plus the
 * body force). */
static void collide_eval(int32_t q, const vlbo_cell *cell, double tau, const double *N,
                         double rho, const double U[3], const double F[3], double *feq,
                         double dPi[3][3], double *dN, double *Om, double *Np, double Fnew[3]) {
  int D = lat_dim(q);
  const int32_t(*c)[3] = lat_c(q);
  const double *w = lat_w(q);
  const double T0 = lat_T0(q);
  double J = cell->J;
  double Ut[3] = {0, 0, 0};
  /* U~ = U + a/2 with rho a = F (text after Eq. 32) */
  for (int i = 0; i < D; i++) Ut[i] = U[i] + 0.5 * (F[i] / rho);
  double ginv[9] = {0};
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) ginv[3 * i + j] = cell->ginv[i][j];
  vlbo_equilibrium(q, rho, U, Ut, ginv, feq);

  /* deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i c^k [Theta^j_k(q+c_a,q) - Theta^j_k(q-c_a,q)] f^eq_a
   * (Eq. 30); q - c_a = q + c_abar */
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) dPi[i][j] = 0.0;
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) {
      double s = 0.0;
      for (int a = 0; a < q; a++) {
        int ab = opposite(q, a);
        for (int k = 0; k < D; k++)
          s += c[a][i] * c[a][k] * (cell->theta[a][j][k] - cell->theta[ab][j][k]) * feq[a];
      }
      dPi[i][j] = -0.5 * (1.0 - 1.0 / (2.0 * tau)) * s;
    }

  for (int a = 0; a < q; a++) {
    /* deltaN_a = w_a J [c^j F^j / T0 + (c^j c^k / T0 - delta^jk) deltaPi^jk / T0]   (Eq. 31) */
    double s = 0.0;
    for (int j = 0; j < D; j++) s += c[a][j] * F[j] / T0;
    for (int j = 0; j < D; j++)
      for (int k = 0; k < D; k++) s += (c[a][j] * c[a][k] / T0 - kd(j, k)) * dPi[j][k] / T0;
    dN[a] = w[a] * J * s;
    /* Omega_a = J M_aa (f_a - f^eq_a), M = -1/tau   (Eq. 20, BGK) */
    double f = N[a] / J;
    Om[a] = J * (-1.0 / tau) * (f - feq[a]);
    /* N'_a = N_a + Omega_a + deltaN_a   (right side of Eq. 12) */
    Np[a] = N[a] + Om[a] + dN[a];
  }

  /* J F^i = -1/2 sum_a c^j_a {Theta^i_j(q+c_a,q) N'_a - Theta^i_j(q-c_a,q) N_a}   (Eq. 27) */
  for (int i = 0; i < 3; i++) Fnew[i] = 0.0;
  for (int i = 0; i < D; i++) {
    double s = 0.0;
    for (int a = 0; a < q; a++) {
      int ab = opposite(q, a);
      for (int j = 0; j < D; j++)
        s += c[a][j] * (cell->theta[a][i][j] * Np[a] - cell->theta[ab][i][j] * N[a]);
    }
    double JF = -0.5 * s;
    Fnew[i] = JF / J + rho * cell->G[i];
  }
}

int vlbo_collide(int32_t q, const vlbo_cell *cell, const vlbo_params *p, const double *N,
                 double *Np_out, double *F_out, double *feq_out, double *dPi_out,
                 double *dN_out, double *Om_out, int32_t *iters_out) {
  if (!lat_known(q)) return VLBO_EINVAL;
  int D = lat_dim(q);
  const int32_t(*c)[3] = lat_c(q);
  double J = cell->J;
  int max_iter = p->max_iter > 0 ? p->max_iter : 200;
  double tol = p->tol > 0.0 ? p->tol : 1e-14;

  /* rho = sum_a f_a, rho U^i = sum_a c^i_a f_a with f = N/J   (Eqs. 14, 15, 17) */
  double rho = 0.0;
  for (int a = 0; a < q; a++) rho += N[a] / J;
  double U[3] = {0, 0, 0};
  for (int i = 0; i < D; i++) {
    double s = 0.0;
    for (int a = 0; a < q; a++) s += c[a][i] * (N[a] / J);
    U[i] = s / rho;
  }

  double feq[VLBO_QMAX], dN[VLBO_QMAX], Om[VLBO_QMAX], Np[VLBO_QMAX], dPi[3][3];
  double F[3] = {0, 0, 0}, Fn[3];
  int it = 0, conv = 0;
  while (it < max_iter) {
    collide_eval(q, cell, p->tau, N, rho, U, F, feq, dPi, dN, Om, Np, Fn);
    it++;
    double diff = 0.0, fmax = 0.0;
    for (int i = 0; i < D; i++) {
      double d = fabs(Fn[i] - F[i]);
      if (d > diff) diff = d;
      if (fabs(Fn[i]) > fmax) fmax = fabs(Fn[i]);
      F[i] = Fn[i];
    }
    double scale = rho > fmax ? rho : fmax;
    if (diff <= tol * scale) {
      conv = 1;
      break;
    }
  }
  if (iters_out) *iters_out = it;
  if (!conv) return VLBO_ENOCONV;
  /* final N' with the converged F */
  collide_eval(q, cell, p->tau, N, rho, U, F, feq, dPi, dN, Om, Np, Fn);
  for (int a = 0; a < q; a++) {
    if (Np_out) Np_out[a] = Np[a];
    if (feq_out) feq_out[a] = feq[a];
    if (dN_out) dN_out[a] = dN[a];
    if (Om_out) Om_out[a] = Om[a];
  }
  if (F_out)
    for (int i = 0; i < 3; i++) F_out[i] = F[i];
  if (dPi_out)
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) dPi_out[3 * i + j] = dPi[i][j];
  return VLBO_OK;
}

/* ------------------------------------------------------------------------- */
/* Whole-mesh simulation. */

struct vlbo_sim {
  vlbo_mesh m;
  double *x;
  vlbo_params p;
  int64_t ncell;
  vlbo_cell *cells;
  double *N, *Nn;
  int32_t last_iters;
};

static void cell_coords(const vlbo_mesh *m, int64_t idx, int64_t q[3]) {
  q[2] = idx % m->n[2];
  int64_t t = idx / m->n[2];
  q[1] = t % m->n[1];
  q[0] = t / m->n[1];
}

int vlbo_create(const vlbo_mesh *m, const vlbo_params *p, vlbo_sim **out) {
  *out = NULL;
  if (!m || !p || !m->x) return VLBO_EINVAL;
  if (!((m->dim == 2 && m->q == 9) || (m->dim == 3 && (m->q == 19 || m->q == 39)))) return VLBO_EINVAL;
  if (m->dim == 2 && m->n[2] != 1) return VLBO_EINVAL;
  for (int a = 0; a < m->dim; a++) {
    if (m->n[a] < 1) return VLBO_EINVAL;
    if (m->bc[a] == VLBO_WALL && m->n[a] < 2) return VLBO_EINVAL;
    /* D3Q39 (speeds up to 3): periodic axes of at least 3 cells only; halfway
     * bounce-back is defined here for links that leave by one cell */
    if (m->q == 39 && (m->bc[a] == VLBO_WALL || m->n[a] < 3)) return VLBO_EINVAL;
  }
  if (!(p->tau > 0.5)) return VLBO_EINVAL;
  vlbo_sim *s = (vlbo_sim *)calloc(1, sizeof(vlbo_sim));
  if (!s) return VLBO_ENOMEM;
  s->m = *m;
  s->p = *p;
  s->ncell = m->n[0] * m->n[1] * m->n[2];
  s->x = (double *)malloc(sizeof(double) * s->ncell * m->dim);
  s->cells = (vlbo_cell *)malloc(sizeof(vlbo_cell) * s->ncell);
  s->N = (double *)calloc(s->ncell * m->q, sizeof(double));
  s->Nn = (double *)calloc(s->ncell * m->q, sizeof(double));
  if (!s->x || !s->cells || !s->N || !s->Nn) {
    vlbo_destroy(s);
    return VLBO_ENOMEM;
  }
  memcpy(s->x, m->x, sizeof(double) * s->ncell * m->dim);
  s->m.x = s->x;
  for (int64_t k = 0; k < s->ncell; k++) {
    int64_t q[3];
    cell_coords(&s->m, k, q);
    int rc = vlbo_cell_geometry(&s->m, &s->p, q, &s->cells[k]);
    if (rc) {
      vlbo_destroy(s);
      return rc;
    }
  }
  *out = s;
  return VLBO_OK;
}

void vlbo_destroy(vlbo_sim *s) {
  if (!s) return;
  free(s->x);
  free(s->cells);
  free(s->N);
  free(s->Nn);
  free(s);
}

int vlbo_init(vlbo_sim *s, const double *rho, const double *u) {
  int q = s->m.q, D = s->m.dim;
  for (int64_t k = 0; k < s->ncell; k++) {
    const vlbo_cell *cl = &s->cells[k];
    double U[3] = {0, 0, 0}, uu[3] = {0, 0, 0}, ginv[9] = {0}, feq[VLBO_QMAX];
    for (int d = 0; d < D; d++) uu[d] = u[k * D + d];
    for (int i = 0; i < D; i++) U[i] = dot3(uu, cl->g_up[i]); /* U^i = u . g^i */
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) ginv[3 * i + j] = cl->ginv[i][j];
    vlbo_equilibrium(q, rho[k], U, U, ginv, feq);
    for (int a = 0; a < q; a++) s->N[a * s->ncell + k] = cl->J * feq[a];
  }
  return VLBO_OK;
}

int vlbo_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* One time step per pass over the cells. Each cell reads only its own
 * arrived populations and writes each of its post-collision populations to a
 * location no other cell writes, so the cells may be taken by several
 * threads (OpenMP) with results identical bit for bit to one thread; a
 * failed solve is reported for the lowest failing cell index. */
int vlbo_step(vlbo_sim *s, int64_t nsteps) {
  int q = s->m.q, D = s->m.dim;
  const int32_t(*c)[3] = lat_c(q);
  int64_t nc = s->ncell;
  int32_t maxit = 0;
  for (int64_t t = 0; t < nsteps; t++) {
    int32_t stepit = 0;
    int64_t bad = -1;
    int badrc = 0;
#pragma omp parallel for schedule(static) reduction(max : stepit)
    for (int64_t k = 0; k < nc; k++) {
      const vlbo_cell *cl = &s->cells[k];
      double N[VLBO_QMAX], Np[VLBO_QMAX];
      for (int a = 0; a < q; a++) N[a] = s->N[a * nc + k];
      int32_t it = 0;
      int rc = vlbo_collide(q, cl, &s->p, N, Np, NULL, NULL, NULL, NULL, NULL, &it);
      if (it > stepit) stepit = it;
      if (rc) {
#pragma omp critical(vlbo_step_error)
        {
          if (bad < 0 || k < bad) {
            bad = k;
            badrc = rc;
          }
        }
        continue;
      }
      double rho = 0.0;
      for (int a = 0; a < q; a++) rho += N[a] / cl->J;
      int64_t qc[3];
      cell_coords(&s->m, k, qc);
      for (int a = 0; a < q; a++) {
        int ab = opposite(q, a);
        if (cl->wall_link[a]) {
          /* halfway bounce-back; a moving wall subtracts J rho (f^eq_a - f^eq_abar) at the
           * wall velocity */
          double ginv[9] = {0}, fw[VLBO_QMAX];
          for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) ginv[3 * i + j] = cl->ginv[i][j];
          vlbo_equilibrium(q, 1.0, cl->uw[a], cl->uw[a], ginv, fw);
          s->Nn[ab * nc + k] = Np[a] - cl->J * rho * (fw[a] - fw[ab]);
          continue;
        }
        /* one-to-one advection N_a(q + c_a, t + 1) = N'_a(q, t)   (Eq. 22) */
        int64_t p[3];
        for (int d = 0; d < 3; d++) {
          p[d] = qc[d] + (d < D ? c[a][d] : 0);
          if (p[d] < 0) p[d] += s->m.n[d];
          if (p[d] >= s->m.n[d]) p[d] -= s->m.n[d];
        }
        s->Nn[a * nc + node_index(&s->m, p)] = Np[a];
      }
    }
    if (stepit > maxit) maxit = stepit;
    if (bad >= 0) {
      s->last_iters = maxit;
      return badrc;
    }
    double *tmp = s->N;
    s->N = s->Nn;
    s->Nn = tmp;
  }
  s->last_iters = maxit;
  return VLBO_OK;
}

int vlbo_moments(vlbo_sim *s, double *rho_out, double *u_out, double *ut_out, double *F_out,
                 double *totals) {
  int q = s->m.q, D = s->m.dim;
  const int32_t(*c)[3] = lat_c(q);
  int64_t nc = s->ncell;
  double tot[7] = {0, 0, 0, 0, 0, 0, 0};
  int32_t maxit = 0;
  for (int64_t k = 0; k < nc; k++) {
    const vlbo_cell *cl = &s->cells[k];
    double N[VLBO_QMAX], F[3];
    for (int a = 0; a < q; a++) N[a] = s->N[a * nc + k];
    int32_t it = 0;
    int rc = vlbo_collide(q, cl, &s->p, N, NULL, F, NULL, NULL, NULL, NULL, &it);
    if (it > maxit) maxit = it;
    if (rc) return rc;
    double rho = 0.0, U[3] = {0, 0, 0}, Ut[3] = {0, 0, 0};
    for (int a = 0; a < q; a++) rho += N[a] / cl->J;
    for (int i = 0; i < D; i++) {
      double sm = 0.0;
      for (int a = 0; a < q; a++) sm += c[a][i] * (N[a] / cl->J);
      U[i] = sm / rho;
      Ut[i] = U[i] + 0.5 * (F[i] / rho);
    }
    if (rho_out) rho_out[k] = rho;
    for (int d = 0; d < D; d++) {
      double uu = 0.0, ut = 0.0;
      for (int i = 0; i < D; i++) {
        uu += U[i] * cl->g_low[i][d]; /* u = U^i g_i   (Eq. 34) */
        ut += Ut[i] * cl->g_low[i][d];
      }
      if (u_out) u_out[k * D + d] = uu;
      if (ut_out) ut_out[k * D + d] = ut;
      if (F_out) F_out[k * D + d] = F[d];
    }
    /* totals: mass, P = sum e_a(q) N_a, M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a */
    int64_t qc[3];
    cell_coords(&s->m, k, qc);
    for (int a = 0; a < q; a++) {
      tot[0] += N[a];
      double e[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
      for (int i = 0; i < D; i++)
        for (int d = 0; d < 3; d++) e[d] += c[a][i] * cl->g_low[i][d];
      int64_t pb[3] = {qc[0] - c[a][0], qc[1] - c[a][1], qc[2] - c[a][2]};
      int across_wall = 0;
      for (int d = 0; d < D; d++)
        if (s->m.bc[d] == VLBO_WALL && (pb[d] < 0 || pb[d] >= s->m.n[d])) across_wall = 1;
      if (across_wall) {
        for (int d = 0; d < 3; d++) eb[d] = e[d];
      } else {
        double gb[3][3];
        tangents(&s->m, pb, gb);
        for (int i = 0; i < D; i++)
          for (int d = 0; d < 3; d++) eb[d] += c[a][i] * gb[i][d];
      }
      for (int d = 0; d < D; d++) {
        tot[1 + d] += e[d] * N[a];
        tot[4 + d] += 0.5 * (e[d] + eb[d]) * N[a];
      }
    }
  }
  if (totals)
    for (int i = 0; i < 7; i++) totals[i] = tot[i];
  s->last_iters = maxit;
  return VLBO_OK;
}

int vlbo_get_state(const vlbo_sim *s, double *N) {
  memcpy(N, s->N, sizeof(double) * s->ncell * s->m.q);
  return VLBO_OK;
}

int vlbo_set_state(vlbo_sim *s, const double *N) {
  memcpy(s->N, N, sizeof(double) * s->ncell * s->m.q);
  return VLBO_OK;
}

int vlbo_get_cell(const vlbo_sim *s, int64_t idx, vlbo_cell *out) {
  if (idx < 0 || idx >= s->ncell) return VLBO_EINVAL;
  *out = s->cells[idx];
  return VLBO_OK;
}

int32_t vlbo_last_iters(const vlbo_sim *s) { return s->last_iters; }

// vlb_q39.cu -- the time step, initialisation, moments and state access for the
// 6th-order isotropic D3Q39 velocity set (vlb_q39.cuh) on periodic meshes, in
// FP64. The reduced force map of the D3Q19/D2Q9 kernels relies on velocity
// components in {-1, 0, 1}; here every relation of section 2.2 is evaluated
// pair of opposite directions by pair instead:
//   f = N / J, rho and U (Eqs. 14, 15, 17); a fixed point on F (Eq. 27), each
//   evaluation forming U~ = U + F / (2 rho), f^eq (Eq. 33 with T0 = 2/3),
//   deltaPi (Eq. 30), deltaN (Eq. 31), Omega = -(N - J f^eq) / tau (Eq. 20)
//   and N' = N + Omega + deltaN (Eq. 12); the converged N' is advected one to
//   one (Eq. 22) in place with the A-A pattern of the other kernels (even
//   steps: slot a of q in, slot abar of q out; odd steps: slot abar of q - c_a
//   in, slot a of q + c_a out), with neighbours wrapped periodically on every
//   axis (each axis at least 3 cells long, speeds at most 3).
// The link coefficients K^i_a = sum_j c^j_a Theta^i_j(q + c_a, q) (Eq. 11)
// come from the mesh's FP64 geometry, so the relations of Eqs. 27 and 30 read
//   sum_j c^j_a Theta^i_j(q - c_a, q) = -K^i_abar.
#include "vlb_addr.cuh"
#include "vlb_q39.cuh"

namespace vlb {
namespace {

constexpr int kQ39 = 39, kH39 = 19;
constexpr int kQ39Threads = 128;

// the velocity set and weights as a table in constant memory: the direction
// loops below are not unrolled, and a warp reads one entry at a time
struct Q39Table {
  double c[kQ39][3];
  double w[kQ39];
};
constexpr Q39Table make_q39_table() {
  Q39Table t{};
  for (int a = 0; a < kQ39; a++) {
    for (int d = 0; d < 3; d++) t.c[a][d] = Lat<39>::c(a, d);
    t.w[a] = q39_w(a);
  }
  return t;
}
__constant__ Q39Table kT39 = make_q39_table();

struct Q39Args {
  double *f;  // populations [39][ncell]
  int64_t ncell;
  int64_t n[3];
  const double *J, *gl, *gu, *ginv, *K;
  // per cell: the chord matrix H = (I - dG/dF)^-1 of the force map at the
  // rest state (row-major) and the rest state's force at rho = 1, 12 values;
  // NULL before q39_prepare has filled them
  const double *chord;
  double body[3];
  double tau, tol;
  int32_t max_iter;
  int *err;
};

__device__ __forceinline__ int opp39(int a) { return a == 0 ? 0 : (a <= kH39 ? a + kH39 : a - kH39); }

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// cell index of q + s c_a (periodic on every axis; |c| <= 3 <= n)
__device__ __forceinline__ int64_t nb39(const Q39Args &A, const int64_t ic[3], int a, int s) {
  const int64_t i0 = wrap(ic[0] + s * Lat<39>::c(a, 0), A.n[0]);
  const int64_t i1 = wrap(ic[1] + s * Lat<39>::c(a, 1), A.n[1]);
  const int64_t i2 = wrap(ic[2] + s * Lat<39>::c(a, 2), A.n[2]);
  return (i0 * A.n[1] + i1) * A.n[2] + i2;
}

__device__ __forceinline__ void coords(const Q39Args &A, int64_t c, int64_t ic[3]) {
  ic[2] = c % A.n[2];
  const int64_t r = c / A.n[2];
  ic[1] = r % A.n[1];
  ic[0] = r / A.n[1];
}

// storage location of the arrived population N_a(q) (A-A)
template <bool ODD>
__device__ __forceinline__ int64_t src39(const Q39Args &A, int64_t c, const int64_t ic[3], int a) {
  if (!ODD || a == 0) return (int64_t)a * A.ncell + c;
  return (int64_t)opp39(a) * A.ncell + nb39(A, ic, a, -1);
}
// storage location that receives N'_a(q)
template <bool ODD>
__device__ __forceinline__ int64_t dst39(const Q39Args &A, int64_t c, const int64_t ic[3], int a) {
  if (!ODD) return (int64_t)opp39(a) * A.ncell + c;
  if (a == 0) return c;
  return (int64_t)a * A.ncell + nb39(A, ic, a, +1);
}

// g^ij - delta^ij of a cell (full 3 x 3) and G^i = G . g^i
__device__ void cell_metric(const Q39Args &A, int64_t c, double gd[3][3], double G[3]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) gd[i][j] = A.ginv[c * 6 + sym<3>(i, j)] - (i == j ? 1.0 : 0.0);
  for (int i = 0; i < 3; i++) {
    double s = 0.0;
    for (int d = 0; d < 3; d++) s += A.body[d] * A.gu[(c * 3 + i) * 3 + d];
    G[i] = s;
  }
}

// The two Hermite tensors of Eq. 33, with B^ij = (g^ij - delta^ij) T0 +
// U~^i U~^j and C^ijk = T0 [(g^ij U~^k - delta^ij U^k) + cyclic] + U~^i U~^j U~^k,
// V^i = C^ijj and tr B, formed once per evaluation
struct Herm39 {
  double B[3][3], C[3][3][3], V[3], trB;
};
__device__ void herm39(const double U[3], const double Ut[3], const double gd[3][3], Herm39 &h) {
  const double T0 = kT0_39;
  h.trB = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) h.B[i][j] = gd[i][j] * T0 + Ut[i] * Ut[j];
  for (int i = 0; i < 3; i++) h.trB += h.B[i][i];
  // g^ij U~^k - delta^ij U^k = gd^ij U~^k + delta^ij (U~^k - U^k)
  auto term = [&](int i, int j, int k) { return gd[i][j] * Ut[k] + (i == j ? Ut[k] - U[k] : 0.0); };
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++)
        h.C[i][j][k] = T0 * (term(i, j, k) + term(j, k, i) + term(k, i, j)) + Ut[i] * Ut[j] * Ut[k];
  for (int i = 0; i < 3; i++) h.V[i] = h.C[i][0][0] + h.C[i][1][1] + h.C[i][2][2];
}

// The bracket of Eq. 33 for direction c split into its even part (the same
// for c and -c) and its odd part (opposite signs):
//   f^eq_{+-c} = rho w {ev +- od},  ev = 1 + (c.B.c / T0 - tr B) / (2 T0),
//   od = c.U / T0 + (C:ccc - 3 T0 c.V) / (6 T0^3),
// with the symmetric contractions over their distinct components (c.B.c from
// 6 terms, C:ccc from 10)
__device__ __forceinline__ void feq39_pair(const Herm39 &h, const double U[3], double x, double y, double z,
                                           double &ev, double &od) {
  const double T0 = kT0_39;
  const double cu = x * U[0] + y * U[1] + z * U[2];
  const double cV = x * h.V[0] + y * h.V[1] + z * h.V[2];
  const double cBc = x * x * h.B[0][0] + y * y * h.B[1][1] + z * z * h.B[2][2] +
                     2.0 * (x * y * h.B[0][1] + x * z * h.B[0][2] + y * z * h.B[1][2]);
  const double cCc = x * x * x * h.C[0][0][0] + y * y * y * h.C[1][1][1] + z * z * z * h.C[2][2][2] +
                     3.0 * (x * x * y * h.C[0][0][1] + x * x * z * h.C[0][0][2] + y * y * x * h.C[1][1][0] +
                            y * y * z * h.C[1][1][2] + z * z * x * h.C[2][2][0] + z * z * y * h.C[2][2][1]) +
                     6.0 * x * y * z * h.C[0][1][2];
  ev = 1.0 + (cBc / T0 - h.trB) / (2.0 * T0);
  od = cu / T0 + (cCc - 3.0 * T0 * cV) / (6.0 * T0 * T0 * T0);
}

// Eq. 33 for every direction (used at set-up and for initialisation)
__device__ void feq39(double rho, const double U[3], const double Ut[3], const double gd[3][3],
                      double f[kQ39]) {
  Herm39 h;
  herm39(U, Ut, gd, h);
  f[0] = rho * kT39.w[0] * (1.0 - h.trB / (2.0 * kT0_39));
#pragma unroll 1
  for (int p = 1; p <= kH39; p++) {
    double ev, od;
    feq39_pair(h, U, kT39.c[p][0], kT39.c[p][1], kT39.c[p][2], ev, od);
    f[p] = rho * kT39.w[p] * (ev + od);
    f[p + kH39] = rho * kT39.w[p] * (ev - od);
  }
}

// One evaluation of the collision at force F (Eqs. 20, 27, 30, 31, 33):
// post-collision N' and the updated F. Directions are taken in pairs
// (p, pbar = p + 19) with c_pbar = -c_p, so each pair's contractions are
// formed once and split into even and odd parts.
__device__ void eval39(const double N[kQ39], double J, double rho, const double U[3], const double F[3],
                       const double gd[3][3], const double G[3], const double *K, double tau,
                       double Np[kQ39], double Fn[3]) {
  const double T0 = kT0_39;
  double Ut[3];
  for (int i = 0; i < 3; i++) Ut[i] = U[i] + 0.5 * (F[i] / rho);
  Herm39 h;
  herm39(U, Ut, gd, h);
  // rho w_p times the even and odd parts of each pair's bracket
  double fe[kH39 + 1], fo[kH39 + 1];
  fe[0] = rho * kT39.w[0] * (1.0 - h.trB / (2.0 * T0));
  fo[0] = 0.0;
  // deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i_a (K^j_a + K^j_abar) f^eq_a   (Eq. 30);
  // over a pair, c_p (K_p + K_pbar) (f^eq_p - f^eq_pbar) = c_p (K_p + K_pbar) 2 rho w_p od_p
  double dP[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll 1
  for (int p = 1; p <= kH39; p++) {
    const double x = kT39.c[p][0], y = kT39.c[p][1], z = kT39.c[p][2];
    double ev, od;
    feq39_pair(h, U, x, y, z, ev, od);
    const double rw = rho * kT39.w[p];
    fe[p] = rw * ev;
    fo[p] = rw * od;
    const double cv[3] = {x, y, z};
    const double d2 = 2.0 * fo[p];
    for (int j = 0; j < 3; j++) {
      const double m = (K[p * 3 + j] + K[(p + kH39) * 3 + j]) * d2;
      for (int i = 0; i < 3; i++) dP[i][j] += cv[i] * m;
    }
  }
  const double cp = -0.5 * (1.0 - 1.0 / (2.0 * tau));
  double tr = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) dP[i][j] *= cp;
  for (int i = 0; i < 3; i++) tr += dP[i][i];
  // c.dP.c over the diagonal and the symmetrised off-diagonal components
  const double s01 = dP[0][1] + dP[1][0], s02 = dP[0][2] + dP[2][0], s12 = dP[1][2] + dP[2][1];
  // deltaN_a = w_a J [c.F / T0 + (c.deltaPi.c / T0 - tr deltaPi) / T0]   (Eq. 31)
  // N'_a = N_a - (N_a - J f^eq_a) / tau + deltaN_a   (Eqs. 12, 20)
  Np[0] = N[0] - (N[0] - J * fe[0]) / tau + kT39.w[0] * J * (-tr / T0);
#pragma unroll 1
  for (int p = 1; p <= kH39; p++) {
    const double x = kT39.c[p][0], y = kT39.c[p][1], z = kT39.c[p][2];
    const double cF = x * F[0] + y * F[1] + z * F[2];
    const double cPc = x * x * dP[0][0] + y * y * dP[1][1] + z * z * dP[2][2] + x * y * s01 + x * z * s02 + y * z * s12;
    const double wJ = kT39.w[p] * J;
    const double dNe = wJ * ((cPc / T0 - tr) / T0), dNo = wJ * (cF / T0);
    const int pb = p + kH39;
    Np[p] = N[p] - (N[p] - J * (fe[p] + fo[p])) / tau + (dNe + dNo);
    Np[pb] = N[pb] - (N[pb] - J * (fe[p] - fo[p])) / tau + (dNe - dNo);
  }
  // J F^i = -1/2 sum_a (K^i_a N'_a + K^i_abar N_a) + J rho G^i   (Eq. 27 and the body force)
  for (int i = 0; i < 3; i++) {
    double s = 0.0;
    for (int a = 1; a < kQ39; a++) s += K[a * 3 + i] * Np[a] + K[opp39(a) * 3 + i] * N[a];
    Fn[i] = -0.5 * s / J + rho * G[i];
  }
}

// The local fixed point on F (Eq. 27 with the body force). With the cell's
// chord data ch: the chord iteration F <- F + H (G(F) - F) from rho F_rest
// (the map is homogeneous of degree one in (N, F) at rest, so rho F_rest is
// the rest state's fixed point at density rho); H inverts the linear part of
// G at rest, so a few evaluations suffice. Without it (ch NULL): the plain
// iteration F <- G(F) from F = 0. Converged when the change is at most
// tol max(rho, |F|); N' at the converged F (to within that change). False if
// max_iter is reached.
__device__ bool collide39(const double N[kQ39], double J, const double gd[3][3], const double G[3],
                          const double *K, const double *ch, double tau, double tol, int max_iter,
                          double Np[kQ39], double &rho, double U[3], double F[3]) {
  rho = 0.0;
  for (int a = 0; a < kQ39; a++) rho += N[a] / J;
  for (int i = 0; i < 3; i++) {
    double s = 0.0;
    for (int a = 0; a < kQ39; a++) s += kT39.c[a][i] * (N[a] / J);
    U[i] = s / rho;
    F[i] = ch ? rho * ch[9 + i] : 0.0;
  }
  bool conv = false;
  double Fn[3];
  for (int it = 0; it < max_iter; it++) {
    eval39(N, J, rho, U, F, gd, G, K, tau, Np, Fn);
    double diff = 0.0, fmax = 0.0;
    if (ch) {
      double r[3];
      for (int i = 0; i < 3; i++) r[i] = Fn[i] - F[i];
      for (int i = 0; i < 3; i++) {
        const double d = ch[3 * i] * r[0] + ch[3 * i + 1] * r[1] + ch[3 * i + 2] * r[2];
        F[i] += d;
        diff = maxnan(diff, fabs(d));
        fmax = maxnan(fmax, fabs(F[i]));
      }
    } else {
      for (int i = 0; i < 3; i++) {
        diff = maxnan(diff, fabs(Fn[i] - F[i]));
        fmax = maxnan(fmax, fabs(Fn[i]));
        F[i] = Fn[i];
      }
    }
    if (diff <= tol * (rho > fmax ? rho : fmax)) {
      conv = true;
      break;
    }
  }
  // N' at the converged F: with the chord iteration the last evaluation was
  // at the F that the final correction, below tol max(rho, |F|), moved off,
  // so its N' is kept; the plain iteration evaluates once more
  if (!(ch && conv)) eval39(N, J, rho, U, F, gd, G, K, tau, Np, Fn);
  return conv;
}

// Chord data of every cell: the rest state N = J f^eq(1, 0) of Eq. 33, its
// force F_rest by the plain iteration (to 1e-15), and the Jacobian of the map
// F -> G(F) there by central differences (G is a cubic polynomial in F, so
// the difference error is of the order of the step squared); H = (I - Jac)^-1.
__global__ void __launch_bounds__(kQ39Threads) k_prep39(const Q39Args A, double *out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double gd[3][3], G[3], U0[3] = {0.0, 0.0, 0.0}, N[kQ39], Np[kQ39], F[3] = {0.0, 0.0, 0.0}, Fn[3];
    cell_metric(A, c, gd, G);
    const double J = A.J[c];
    feq39(1.0, U0, U0, gd, N);
    for (int a = 0; a < kQ39; a++) N[a] *= J;
    const double *K = A.K + c * kQ39 * 3;
    for (int it = 0; it < 400; it++) {
      eval39(N, J, 1.0, U0, F, gd, G, K, A.tau, Np, Fn);
      double diff = 0.0, fm = 0.0;
      for (int i = 0; i < 3; i++) {
        diff = maxnan(diff, fabs(Fn[i] - F[i]));
        fm = maxnan(fm, fabs(Fn[i]));
        F[i] = Fn[i];
      }
      if (diff <= 1e-15 * (fm > 1.0 ? fm : 1.0)) break;
    }
    double Jac[3][3];
    const double h = 1e-6;
    for (int j = 0; j < 3; j++) {
      double Fp[3] = {F[0], F[1], F[2]}, Fm[3] = {F[0], F[1], F[2]}, Gp[3], Gm[3];
      Fp[j] += h;
      Fm[j] -= h;
      eval39(N, J, 1.0, U0, Fp, gd, G, K, A.tau, Np, Gp);
      eval39(N, J, 1.0, U0, Fm, gd, G, K, A.tau, Np, Gm);
      for (int i = 0; i < 3; i++) Jac[i][j] = (Gp[i] - Gm[i]) / (2.0 * h);
    }
    double M[3][3], C[3][3];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) M[i][j] = (i == j ? 1.0 : 0.0) - Jac[i][j];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        C[i][j] = M[i1][j1] * M[i2][j2] - M[i1][j2] * M[i2][j1];
      }
    const double det = M[0][0] * C[0][0] + M[0][1] * C[0][1] + M[0][2] * C[0][2];
    double *o = out + c * 12;
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) o[3 * i + j] = C[j][i] / det;
    for (int i = 0; i < 3; i++) o[9 + i] = F[i];
  }
}

template <bool ODD>
__global__ void __launch_bounds__(kQ39Threads) k_step39(const Q39Args A) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t ic[3];
    coords(A, c, ic);
    double N[kQ39], Np[kQ39];
#pragma unroll 1
    for (int a = 0; a < kQ39; a++) N[a] = A.f[src39<ODD>(A, c, ic, a)];
    double gd[3][3], G[3], rho, U[3], F[3];
    cell_metric(A, c, gd, G);
    if (!collide39(N, A.J[c], gd, G, A.K + c * kQ39 * 3, A.chord ? A.chord + c * 12 : nullptr, A.tau, A.tol,
                   A.max_iter, Np, rho, U, F))
      atomicOr(A.err, ERR_NOCONV);
#pragma unroll 1
    for (int a = 0; a < kQ39; a++) A.f[dst39<ODD>(A, c, ic, a)] = Np[a];
  }
}

__global__ void __launch_bounds__(kQ39Threads) k_init39(const Q39Args A, const double *rho, const double *u) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double gd[3][3], G[3], U[3], f[kQ39];
    cell_metric(A, c, gd, G);
    for (int i = 0; i < 3; i++) {
      double s = 0.0;
      for (int d = 0; d < 3; d++) s += u[c * 3 + d] * A.gu[(c * 3 + i) * 3 + d];  // U^i = u . g^i
      U[i] = s;
    }
    feq39(rho[c], U, U, gd, f);
    const double J = A.J[c];
    for (int a = 0; a < kQ39; a++) A.f[(int64_t)a * A.ncell + c] = J * f[a];
  }
}

__device__ __forceinline__ double warp_sum39(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// rho [ncell], u [ncell][3], u~ [ncell][3] into out; per-block conservation
// sums (mass, P = sum e_a N_a, M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a) into
// partial[block][7]
template <bool ODD>
__global__ void __launch_bounds__(kMomThreads) k_moments39(const Q39Args A, double *out, double *partial) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t ic[3];
    coords(A, c, ic);
    double N[kQ39], Np[kQ39];
#pragma unroll 1
    for (int a = 0; a < kQ39; a++) N[a] = A.f[src39<ODD>(A, c, ic, a)];
    double gd[3][3], G[3], rho, U[3], F[3];
    cell_metric(A, c, gd, G);
    if (!collide39(N, A.J[c], gd, G, A.K + c * kQ39 * 3, A.chord ? A.chord + c * 12 : nullptr, A.tau, A.tol,
                   A.max_iter, Np, rho, U, F))
      atomicOr(A.err, ERR_NOCONV);
    const double *gl = A.gl + c * 9;
    out[c] = rho;
    bool finite = isfinite(rho);
    for (int d = 0; d < 3; d++) {
      double uu = 0.0, ut = 0.0;
      for (int i = 0; i < 3; i++) {
        uu += U[i] * gl[i * 3 + d];                          // u = U^i g_i (Eq. 34)
        ut += (U[i] + 0.5 * (F[i] / rho)) * gl[i * 3 + d];   // u~ = U~^i g_i
      }
      out[A.ncell + c * 3 + d] = uu;
      out[A.ncell * 4 + c * 3 + d] = ut;
      finite = finite && isfinite(uu) && isfinite(ut);
    }
    if (!finite) atomicOr(A.err, ERR_NONFINITE);
#pragma unroll 1
    for (int a = 0; a < kQ39; a++) {
      acc[0] += N[a];
      const double *gb = A.gl + nb39(A, ic, a, -1) * 9;
      for (int d = 0; d < 3; d++) {
        double e = 0.0, eb = 0.0;
        for (int i = 0; i < 3; i++) {
          e += Lat<39>::c(a, i) * gl[i * 3 + d];
          eb += Lat<39>::c(a, i) * gb[i * 3 + d];
        }
        acc[1 + d] += e * N[a];
        acc[4 + d] += 0.5 * (e + eb) * N[a];
      }
    }
  }
  __shared__ double sh[7][kMomThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 7; k++) {
    const double s = warp_sum39(acc[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < 7; k++) {
      double s = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
      s = warp_sum39(s);
      if (lane == 0) partial[(int64_t)blockIdx.x * 7 + k] = s;
    }
  }
}

template <bool ODD>
__global__ void k_get39(const Q39Args A, double *N_out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t ic[3];
    coords(A, c, ic);
    for (int a = 0; a < kQ39; a++) N_out[(int64_t)a * A.ncell + c] = A.f[src39<ODD>(A, c, ic, a)];
  }
}

template <bool ODD>
__global__ void k_set39(const Q39Args A, const double *N_in) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t ic[3];
    coords(A, c, ic);
    for (int a = 0; a < kQ39; a++) A.f[src39<ODD>(A, c, ic, a)] = N_in[(int64_t)a * A.ncell + c];
  }
}

// per block: [min J, -max J, min f^eq_rest / w, min g^ii, -max g^ii]
__global__ void __launch_bounds__(kStatThreads) k_stats39(const double *J, const double *ginv, int64_t ncell,
                                                         double *partial) {
  double v[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double gd[3][3], U0[3] = {0, 0, 0}, f[kQ39];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) gd[i][j] = ginv[c * 6 + sym<3>(i, j)] - (i == j ? 1.0 : 0.0);
    feq39(1.0, U0, U0, gd, f);
    v[0] = fmin(v[0], J[c]);
    v[1] = fmin(v[1], -J[c]);
    for (int a = 0; a < kQ39; a++) v[2] = fmin(v[2], f[a] / q39_w(a));
    for (int i = 0; i < 3; i++) {
      const double g = ginv[c * 6 + sym<3>(i, i)];
      v[3] = fmin(v[3], g);
      v[4] = fmin(v[4], -g);
    }
  }
  __shared__ double sh[5][kStatThreads];
  for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; k++) {
      double m = sh[k][0];
      for (int t = 1; t < (int)blockDim.x; t++) m = fmin(m, sh[k][t]);
      partial[(int64_t)blockIdx.x * 5 + k] = m;
    }
  }
}

Q39Args make_args(const vlb_sim *sim) {
  const vlb_mesh *m = sim->mesh;
  Q39Args A;
  A.f = static_cast<double *>(sim->d_f);
  A.ncell = m->ncell;
  for (int d = 0; d < 3; d++) {
    A.n[d] = m->md.n[d];
    A.body[d] = sim->p.body_force[d];
  }
  A.J = m->d_J;
  A.gl = m->d_gl;
  A.gu = m->d_gu;
  A.ginv = m->d_ginv;
  A.K = m->d_K;
  A.chord = static_cast<const double *>(sim->d_coef);
  A.tau = sim->p.tau;
  A.tol = sim->p.tol;
  A.max_iter = sim->p.max_iter;
  A.err = sim->d_err;
  return A;
}

unsigned grid_for(int64_t ncell, int threads) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (ncell + threads - 1) / threads;
  const int64_t cap = (int64_t)nsm * 16;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t q39_mesh_stats(const vlb_mesh *m, double *d_partial, int64_t nblk, cudaStream_t s) {
  k_stats39<<<(unsigned)nblk, kStatThreads, 0, s>>>(m->d_J, m->d_ginv, m->ncell, d_partial);
  return cudaGetLastError();
}

cudaError_t q39_prepare(const vlb_sim *sim, cudaStream_t s) {
  Q39Args A = make_args(sim);
  A.chord = nullptr;
  k_prep39<<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A, static_cast<double *>(sim->d_coef));
  return cudaGetLastError();
}

cudaError_t q39_init(const vlb_sim *sim, const double *d_rho, const double *d_u, cudaStream_t s) {
  const Q39Args A = make_args(sim);
  k_init39<<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A, d_rho, d_u);
  return cudaGetLastError();
}

cudaError_t q39_step(const vlb_sim *sim, int odd, cudaStream_t s) {
  const Q39Args A = make_args(sim);
  if (odd)
    k_step39<true><<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A);
  else
    k_step39<false><<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t q39_moments(const vlb_sim *sim, double *d_out, double *d_partial, int64_t nblk, cudaStream_t s) {
  const Q39Args A = make_args(sim);
  if (sim->t & 1)
    k_moments39<true><<<(unsigned)nblk, kMomThreads, 0, s>>>(A, d_out, d_partial);
  else
    k_moments39<false><<<(unsigned)nblk, kMomThreads, 0, s>>>(A, d_out, d_partial);
  return cudaGetLastError();
}

cudaError_t q39_get_state(const vlb_sim *sim, double *d_N, cudaStream_t s) {
  const Q39Args A = make_args(sim);
  if (sim->t & 1)
    k_get39<true><<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A, d_N);
  else
    k_get39<false><<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A, d_N);
  return cudaGetLastError();
}

// written in the layout of time 0 (even), which the caller then sets
cudaError_t q39_set_state(const vlb_sim *sim, const double *d_N, cudaStream_t s) {
  const Q39Args A = make_args(sim);
  k_set39<false><<<grid_for(A.ncell, kQ39Threads), kQ39Threads, 0, s>>>(A, d_N);
  return cudaGetLastError();
}

}  // namespace vlb

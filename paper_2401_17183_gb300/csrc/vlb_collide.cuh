// vlb_collide.cuh -- the local part of one time step for one cell (section 2.2):
// moments (Eqs. 14, 15, 17), the implicit inertial force F (Eq. 27, with
// deltaPi of Eq. 30 and deltaN of Eq. 31), the curvilinear equilibrium
// (Eq. 33) with U~ = U + F/(2 rho), and the BGK post-collision populations
// N' = N + Omega + deltaN (Eqs. 12, 20). Shared by the step, moments and
// coefficient-packing kernels.
//
// Populations enter and leave as deviations d_a = N_a - w_a n_ref from a
// uniform reference n_ref = rho_0 J_ref (n_ref = 0 gives plain populations).
// The reference is the same in every cell, so advection and bounce-back move
// deviations exactly as they move populations, while every product below
// works on small numbers: that keeps FP32 rounding relative to the deviation,
// not to N. The force is carried as Phi = J F.
//
// Directions come in pairs (p, pbar = p + H) with c_pbar = -c_p; every sum over
// directions is a sum over pairs of an even part (same for p and pbar) and an
// odd part (opposite signs), with the link coefficients stored as
// M_p = K_p + K_pbar and D_p = K_p - K_pbar (stored with the weights they
// carry in the constant part of the map).
//
// The map Phi -> Phi_new of Eq. 27 is evaluated in a reduced form. Writing
//   N'_a - w_a n_ref = (1 - 1/tau) d_a + w_a (mdev + m x_a)/tau + deltaN_a,
// with J f^eq_a = w_a m (1 + x_a) and x_p = xe_p + xo_p, x_pbar = xe_p - xo_p,
// deltaN_p = E_p + O_p, deltaN_pbar = E_p - O_p (Eq. 31, 1/T0 = 3),
//   E_p = 3 w_p J (3 c_p.S.c_p - tr S),  O_p = 3 w_p c_p.Phi,
// S the symmetric part of deltaPi (Eq. 30), linear in the xo_q, gives
//   Phi_new = Pb - 1/2 { m [sum_p Ae_p xe_p + sum_p Ao_p xo_p] + T Phi },
// where Pb holds everything fixed during the iteration. Because xe_p is
// linear in B = gd T0 + U~ U~ and xo_p linear in U and in C^kkl (k != l),
// the pair sums collapse into a polynomial in U~ with per-cell constant
// coefficients (build_record):
//   Phi_new = Pb' - 1/2 { m [PE : U~U~ + PO2 : (U~^k)^2 U~^l + LO U~] + TL Phi },
//   Pb' = Pb - 1/2 m (CE + PO1 U).
// The post-collision populations themselves are formed once, at the converged
// Phi, direction by direction.
//
// In FP32, pairs of identical operations run in the two lanes of packed FP32
// instructions (sm_100 and later): a direction pair (p, pbar) of the final
// pass, rows 0 and 1 of the map and of the chord correction, and components 0
// and 1 of the constant part, each pair with the same roundings in the same
// order as two scalar operations.
#pragma once

#include "vlb_internal.cuh"

namespace vlb {

template <int Q, typename R>
struct CollideState {
  static constexpr int D = Lat<Q>::D;
  R rho;
  R U[D];
  R F[D];
  int iters;
  bool conv;
};

// D x D inverse (D = 2 or 3) by cofactors, FP64
template <int D>
__device__ void inverse_small(const double (&A)[D][D], double (&X)[D][D]) {
  if (D == 2) {
    const double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    X[0][0] = A[1][1] / det;
    X[0][1] = -A[0][1] / det;
    X[1][0] = -A[1][0] / det;
    X[1][1] = A[0][0] / det;
  } else {
    double C[D][D];
    for (int i = 0; i < D; i++)
      for (int j = 0; j < D; j++) {
        const int i1 = (i + 1) % D, i2 = (i + 2) % D, j1 = (j + 1) % D, j2 = (j + 2) % D;
        C[i][j] = A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1];
      }
    double det = 0.0;
    for (int j = 0; j < D; j++) det += A[0][j] * C[0][j];
    for (int i = 0; i < D; i++)
      for (int j = 0; j < D; j++) X[i][j] = C[j][i] / det;
  }
}

// Coefficient record of one cell in FP64 from its geometry: J, g^ij (packed),
// G^i = G . g^i and the link coefficients K^i_a (Eq. 25). Every entry is
// filled except FR and UW, which are left zero. With itau = 1/tau,
// cpi = -(1 - itau/2) and the pair sums over p = 1..H:
//   R^i_kl  = sum_p w_p M^i_p (3 c^k_p c^l_p - delta_kl)
//   Ao^i_p  = w_p [itau D^i_p + 3 cpi c_p.R^i.M_p]    (xo_p: BGK part and, via S, E_p)
//   PE^i_kl = (3/2) itau R^i_kl                        (xe_p: BGK part)
//   PO1^i_l = 3 sum_p Ao^i_p c^l_p
//   PO2^i_kl = (9/2) sum_p Ao^i_p c^l_p (3 (c^k_p)^2 - 1),  k != l
//   TT^i_j  = 3 sum_p w_p D^i_p c^j_p                  (O_p)
//   LO^i_j  = T0 [sum_{k != j} PO2^i_kj gd_kk + 2 sum_{l != j} PO2^i_jl gd_jl]
//   LD^i_j  = T0 sum_{k != j} PO2^i_kj,   TL = TT + LD / 2
//   CE^i    = T0 sum_kl PE^i_kl gd_kl
// and the chord matrix (I - L)^-1 with L = -(LO/4 + TL/2), the part of the
// Jacobian of the map that stays when U -> 0. PE is stored packed over
// k <= l with the off-diagonal entries doubled (U~U~ is symmetric).
template <int Q>
__device__ void build_record(double J, const double *ginv, const double *G,
                             const double (&K)[Q][Lat<Q>::D], double tau, double *rec) {
  using L = CoefLayout<Q>;
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H, NS = L::NS;
  const double T0 = kT0, itau = 1.0 / tau, cpi = -(1.0 - 0.5 * itau);
  for (int k = 0; k < L::NC; k++) rec[k] = 0.0;
  rec[L::J] = J;
  rec[L::IJ] = 1.0 / J;
  double gd[D][D];
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) gd[i][j] = ginv[sym<D>(i, j)] - (i == j ? 1.0 : 0.0);
  for (int i = 0; i < D; i++)
    for (int j = i; j < D; j++) rec[L::GINV + sym<D>(i, j)] = gd[i][j];
  for (int i = 0; i < D; i++) {
    rec[L::BODY + i] = G[i];
    double s = 0.0;
    for (int a = 1; a < Q; a++) s += lat_w<Q, double>(a) * K[a][i];
    rec[L::KW + i] = s;
  }
  double M[H + 1][D], Dk[H + 1][D], c[H + 1][D], w[H + 1];
  for (int p = 1; p <= H; p++) {
    w[p] = lat_w<Q, double>(p);
    for (int i = 0; i < D; i++) {
      M[p][i] = K[p][i] + K[p + H][i];
      Dk[p][i] = K[p][i] - K[p + H][i];
      c[p][i] = Lat<Q>::c(p, i);
      // stored with the weights they carry in the constant part of the map
      rec[L::mp(p, i)] = -0.25 * (2.0 - itau) * M[p][i];
      rec[L::dk(p, i)] = 0.25 * itau * Dk[p][i];
    }
  }
  double Rt[D][D][D];
  for (int i = 0; i < D; i++)
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        double s = 0.0;
        for (int p = 1; p <= H; p++)
          s += w[p] * M[p][i] * (3.0 * c[p][k] * c[p][l] - (k == l ? 1.0 : 0.0));
        Rt[i][k][l] = s;
      }
  double Ao[H + 1][D];
  for (int p = 1; p <= H; p++)
    for (int i = 0; i < D; i++) {
      double cRM = 0.0;
      for (int k = 0; k < D; k++)
        for (int l = 0; l < D; l++) cRM += c[p][k] * Rt[i][k][l] * M[p][l];
      Ao[p][i] = w[p] * (itau * Dk[p][i] + 3.0 * cpi * cRM);
    }
  double PO2[D][D][D];  // [i][k][l]
  double LO[D][D], TL[D][D];
  for (int i = 0; i < D; i++) {
    double ce = 0.0;
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        const double pe = 1.5 * itau * Rt[i][k][l];
        ce += T0 * pe * gd[k][l];
        if (k <= l) rec[L::row(L::PE, NS, i, sym<D>(k, l))] = (k == l ? 1.0 : 2.0) * pe;
      }
    rec[L::CE + i] = ce;
    for (int l = 0; l < D; l++) {
      double s = 0.0;
      for (int p = 1; p <= H; p++) s += Ao[p][i] * c[p][l];
      rec[L::PO1 + i * D + l] = 3.0 * s;
    }
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        PO2[i][k][l] = 0.0;
        if (k == l) continue;
        double s = 0.0;
        for (int p = 1; p <= H; p++) s += Ao[p][i] * c[p][l] * (3.0 * c[p][k] * c[p][k] - 1.0);
        PO2[i][k][l] = 4.5 * s;
        rec[L::row(L::PO2, L::NO, i, offd<D>(k, l))] = PO2[i][k][l];
      }
  }
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) {
      double tt = 0.0;
      for (int p = 1; p <= H; p++) tt += 3.0 * w[p] * Dk[p][i] * c[p][j];
      double lo = 0.0, ld = 0.0;
      for (int k = 0; k < D; k++) {
        if (k == j) continue;
        lo += T0 * (PO2[i][k][j] * gd[k][k] + 2.0 * PO2[i][j][k] * gd[j][k]);
        ld += T0 * PO2[i][k][j];
      }
      LO[i][j] = lo;
      TL[i][j] = tt + 0.5 * ld;
      rec[L::row(L::LO, D, i, j)] = lo;
      rec[L::row(L::TL, D, i, j)] = TL[i][j];
    }
  double A[D][D], Hm[D][D];
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) A[i][j] = (i == j ? 1.0 : 0.0) + 0.25 * LO[i][j] + 0.5 * TL[i][j];
  inverse_small<D>(A, Hm);
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) rec[L::row(L::HM, D, i, j)] = Hm[i][j];
}

// x y = p + e exactly (FMA two-product)
__device__ __forceinline__ float two_prod_err(float x, float y, float p) { return fmaf(x, y, -p); }
__device__ __forceinline__ double two_prod_err(double x, double y, double p) { return fma(x, y, -p); }

// Post-collision deviations dp_a = N'_a - w_a n_ref at a given Phi:
//   N'_a = N_a + Omega_a + deltaN_a, Omega_a = -(N_a - J f^eq_a)/tau (Eqs. 12, 20),
//   N_a - J f^eq_a = (d_a - w_a mdev) - w_a m x_a,
// with the non-equilibrium part formed first, so that its rounding error is
// relative to itself and not to the much larger d_a.
template <int Q, typename R>
__device__ __forceinline__ void form_np(const R (&d)[Q], const R *__restrict__ rc, R m, R mdev,
                                        R h2m, R rho, R itau, const R (&U)[Lat<Q>::D],
                                        const R (&Phi)[Lat<Q>::D], R (&dp)[Q]) {
  using L = CoefLayout<Q>;
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  R gd[L::NS], dU[D];
#pragma unroll
  for (int i = 0; i < L::NS; i++) gd[i] = rc[L::GINV + i];
#pragma unroll
  for (int i = 0; i < D; i++) dU[i] = Phi[i] * h2m;
  // The even and odd parts of the bracket of Eq. 33 divided by 3 (the factor
  // moves into the per-weight constants below), from B and C^kkl of eq_parts
  // scaled by 3/2 (with T0 = 1/3):
  //   xe_p / 3 = c_p.Bh.c_p - tr Bh / 3,   Bh = (3/2) B,
  //   xo_p / 3 = c_p.U + sum_{k != l} C2h^kl c^l_p (3 (c^k_p)^2 - 1),   C2h = (3/2) C^kkl.
  const R hT0 = R(1.5 * kT0);
  R Ut[D], Uh[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    Ut[i] = U[i] + dU[i];
    Uh[i] = R(1.5) * Ut[i];
  }
  R Bh[D][D], tB3 = R(0);
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = i; j < D; j++) {
      Bh[i][j] = gd[sym<D>(i, j)] * hT0 + Uh[i] * Ut[j];
      Bh[j][i] = Bh[i][j];
    }
#pragma unroll
  for (int i = 0; i < D; i++) tB3 += Bh[i][i];
  tB3 *= R(1.0 / 3.0);
  R C2h[D][D];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) {
      if (i == j) continue;
      C2h[i][j] = hT0 * ((gd[sym<D>(i, i)] * Ut[j] + dU[j]) + R(2) * gd[sym<D>(i, j)] * Ut[i]) +
                  Uh[i] * Ut[i] * Ut[j];
    }
  R xe[H + 1], xo[H + 1];
  xe[0] = -tB3;
#pragma unroll
  for (int p = 1; p <= H; p++) {
    R cbc = R(0), x = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci == 0) continue;
      x += ci > 0 ? U[i] : -U[i];
#pragma unroll
      for (int j = 0; j < D; j++) {
        const int cj = Lat<Q>::c(p, j);
        if (cj != 0) cbc += ci * cj > 0 ? Bh[i][j] : -Bh[i][j];
        // 3 (c^j)^2 - 1 is 2 for an in-plane j and -1 otherwise
        if (j != i) x += R((cj != 0 ? 2 : -1) * ci) * C2h[j][i];
      }
    }
    xe[p] = cbc - tB3;
    xo[p] = x;
  }
  // deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i_a (K^j_a - L^j_a) f^eq_a   (Eq. 30):
  // K_a - L_a = K_a + K_abar = M_p, and a pair contributes c_p (f_p - f_pbar)
  // with f_p - f_pbar = 2 rho w_p xo_p = 6 rho w_p (xo_p / 3). The record holds
  // am M_p with am = -(2 - 1/tau)/4, and -1/2 (1 - 1/(2 tau)) 2 rho = 2 rho am.
  const R r6 = R(6) * rho;
  R dP[D][D];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) dP[i][j] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const R df = r6 * lat_w<Q, R>(p) * xo[p];
#pragma unroll
    for (int j = 0; j < D; j++) {
      const R amM = rc[L::mp(p, j)];
#pragma unroll
      for (int i = 0; i < D; i++) {
        const int ci = Lat<Q>::c(p, i);
        if (ci > 0) dP[i][j] = fmar(amM, df, dP[i][j]);
        if (ci < 0) dP[i][j] = fmar(-amM, df, dP[i][j]);
      }
    }
  }
  R tr = R(0);
#pragma unroll
  for (int i = 0; i < D; i++) tr += dP[i][i];
  const R J = rc[L::J];
  {
    const R w = lat_w<Q, R>(0);
    const R neq = (d[0] - w * mdev) - (R(3) * w * m) * xe[0];
    dp[0] = d[0] - itau * neq - (R(3) * w * J) * tr;
  }
#pragma unroll
  for (int p = 1; p <= H; p++) {
    R cF = R(0), cPc = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci == 0) continue;
      cF += ci > 0 ? Phi[i] : -Phi[i];
#pragma unroll
      for (int j = 0; j < D; j++) {
        const int cj = Lat<Q>::c(p, j);
        if (cj == 0) continue;
        cPc += ci * cj > 0 ? dP[i][j] : -dP[i][j];
      }
    }
    const R w = lat_w<Q, R>(p);
    const R Ep = (R(9) * w * J) * cPc - (R(3) * w * J) * tr;
    const R Op = (R(3) * w) * cF;
    const R wd = w * mdev, wm = (R(3) * w) * m;
    if constexpr (sizeof(R) == 4) {
      // the pair in the two lanes of packed FP32 instructions (same roundings)
      const float2 dd = make_float2(d[p], d[p + H]);
      const float2 xs = __fadd2_rn(make_float2(xe[p], xe[p]), make_float2(xo[p], -xo[p]));
      const float2 nq = __ffma2_rn(make_float2(-wm, -wm), xs, __fadd2_rn(dd, make_float2(-wd, -wd)));
      const float2 r = __fadd2_rn(__ffma2_rn(make_float2(-itau, -itau), nq, dd),
                                  __fadd2_rn(make_float2(Ep, Ep), make_float2(Op, -Op)));
      dp[p] = r.x;
      dp[p + H] = r.y;
    } else {
      const R neqp = (d[p] - wd) - wm * (xe[p] + xo[p]);
      const R neqm = (d[p + H] - wd) - wm * (xe[p] - xo[p]);
      dp[p] = d[p] - itau * neqp + (Ep + Op);
      dp[p + H] = d[p + H] - itau * neqm + (Ep - Op);
    }
  }
}

// Full local collision: solve Phi = J G(Phi / J) by a chord iteration
//   Phi <- Phi + H (Phi_new - Phi),  H = (I - L)^-1,
// where L is the part of the Jacobian of the map that does not vanish with
// U (the remainder is of order |U~| times the coefficients, so each chord
// step shrinks the error by about that factor). With CHORD = false, H = I
// (plain fixed-point iteration) and the start value is Phi = 0; with CHORD,
// the start value is m times the rest-state force. A correction is accepted
// as converged when it is at most max(tol max(m, |Phi|), 64 eps |Phi|): eps
// is the unit roundoff of R, and Phi is a sum of dozens of rounded terms of
// its own size, so smaller corrections are rounding noise. With FINAL, the
// post-collision deviations are formed at the converged Phi.
// rc points at the cell's coefficient record (global, shared or local
// memory); itau = 1/tau.
template <int Q, typename R, bool CHORD, bool FINAL>
__device__ __forceinline__ void collide_cell(const R (&d)[Q], const R *__restrict__ rc, R nref,
                                             R itau, R tol, int max_iter, R (&dp)[Q],
                                             CollideState<Q, R> &st) {
  using L = CoefLayout<Q>;
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H, NS = L::NS;
  const R epsn = sizeof(R) == 4 ? R(64.0 / 16777216.0) : R(64.0 / 9007199254740992.0);
  // pair sums s_p = d_p + d_pbar and differences t_p = d_p - d_pbar
  R sp[H + 1], tp[H + 1];
  R mdev = d[0];
#pragma unroll
  for (int p = 1; p <= H; p++) {
    sp[p] = d[p] + d[p + H];
    tp[p] = d[p] - d[p + H];
    mdev += sp[p];
  }
  const R m = nref + mdev;
  // rho = sum f = sum N / J; rho U = sum c f   (Eqs. 14, 15, 17)
  st.rho = m * rc[L::IJ];
  const R im = R(1) / m;
  const R h2m = R(0.5) * im;
#pragma unroll
  for (int i = 0; i < D; i++) {
    R s = R(0);
#pragma unroll
    for (int p = 1; p <= H; p++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci > 0) s += tp[p];
      if (ci < 0) s -= tp[p];
    }
    st.U[i] = s * im;
  }
  // constant part of J F: body force m G, 1/2 sum_a L_a N_a (L_a = -K_abar), the
  // reference part -n_ref sum_a w_a K_a of both sums of Eq. 27 (the largest term,
  // the same every step: formed without rounding error from the split KW + KWL),
  // the parts of -1/2 sum_a K_a N'_a that do not change during the iteration
  // and the terms of the map that depend on U only. Over a pair,
  //   -1/2 (K_pbar d_p + K_p d_pbar) - 1/2 (1 - 1/tau)(K_p d_p + K_pbar d_pbar)
  //     = -(2 - 1/tau)/4 M_p s_p + (1/tau)/4 D_p t_p,
  // whose two weights the record's link coefficients already carry.
  R Pb[D], s[D], pr[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    const R kw = rc[L::KW + i];
    pr[i] = nref * kw;
    const R err = two_prod_err(nref, kw, pr[i]) + nref * rc[L::KWL + i];
    s[i] = m * rc[L::BODY + i] - err - R(0.5) * itau * mdev * kw;
  }
  int ipb = 0;
  if constexpr (sizeof(R) == 4) {
    // components 0 and 1 in the two lanes of packed FP32 instructions (the
    // same roundings in the same order)
    float2 s01 = make_float2(s[0], s[1]);
#pragma unroll
    for (int p = 1; p <= H; p++) {
      s01 = __ffma2_rn(*reinterpret_cast<const float2 *>(rc + L::mp(p, 0)), make_float2(sp[p], sp[p]), s01);
      s01 = __ffma2_rn(*reinterpret_cast<const float2 *>(rc + L::dk(p, 0)), make_float2(tp[p], tp[p]), s01);
    }
    s[0] = s01.x;
    s[1] = s01.y;
    ipb = 2;
  }
#pragma unroll
  for (int i = 0; i < D; i++) {
    if (i < ipb) continue;
#pragma unroll
    for (int p = 1; p <= H; p++) s[i] = fmar(rc[L::dk(p, i)], tp[p], fmar(rc[L::mp(p, i)], sp[p], s[i]));
  }
#pragma unroll
  for (int i = 0; i < D; i++) {
    R u = rc[L::CE + i];
#pragma unroll
    for (int l = 0; l < D; l++) u += rc[L::PO1 + i * D + l] * st.U[l];
    Pb[i] = (s[i] - R(0.5) * m * u) - pr[i];
  }
  R Phi[D];
#pragma unroll
  for (int i = 0; i < D; i++) Phi[i] = CHORD ? m * rc[L::FR + i] : R(0);
  st.conv = false;
  int it = 0;
  while (it < max_iter) {
    // Phi_new = Pb' - 1/2 { m [PE : U~U~ + PO2 : (U~^k)^2 U~^l + LO U~] + TL Phi }
    R Ut[D], Ut2[D];
#pragma unroll
    for (int i = 0; i < D; i++) {
      Ut[i] = st.U[i] + Phi[i] * h2m;
      Ut2[i] = Ut[i] * Ut[i];
    }
    R UU[NS];
#pragma unroll
    for (int k = 0; k < D; k++)
#pragma unroll
      for (int l = k; l < D; l++) UU[sym<D>(k, l)] = Ut[k] * Ut[l];
    R r[D];
    int i0 = 0;
    if constexpr (sizeof(R) == 4) {
      // rows 0 and 1 in the two lanes of packed FP32 instructions
      auto ld2 = [&](int idx) { return *reinterpret_cast<const float2 *>(rc + idx); };
      auto bc = [](float v) { return make_float2(v, v); };
      float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < NS; s++) a = __ffma2_rn(ld2(L::row(L::PE, NS, 0, s)), bc(UU[s]), a);
#pragma unroll
      for (int k = 0; k < D; k++)
#pragma unroll
        for (int l = 0; l < D; l++) {
          if (k == l) continue;
          a = __ffma2_rn(ld2(L::row(L::PO2, L::NO, 0, offd<D>(k, l))), bc(Ut2[k] * Ut[l]), a);
        }
#pragma unroll
      for (int j = 0; j < D; j++) a = __ffma2_rn(ld2(L::row(L::LO, D, 0, j)), bc(Ut[j]), a);
#pragma unroll
      for (int j = 0; j < D; j++) b = __ffma2_rn(ld2(L::row(L::TL, D, 0, j)), bc(Phi[j]), b);
      r[0] = (Pb[0] - R(0.5) * (m * a.x + b.x)) - Phi[0];
      r[1] = (Pb[1] - R(0.5) * (m * a.y + b.y)) - Phi[1];
      i0 = 2;
    }
#pragma unroll
    for (int i = 0; i < D; i++) {
      if (i < i0) continue;
      R a = R(0);
#pragma unroll
      for (int s = 0; s < NS; s++) a += rc[L::row(L::PE, NS, i, s)] * UU[s];
#pragma unroll
      for (int k = 0; k < D; k++)
#pragma unroll
        for (int l = 0; l < D; l++) {
          if (k == l) continue;
          a += rc[L::row(L::PO2, L::NO, i, offd<D>(k, l))] * (Ut2[k] * Ut[l]);
        }
#pragma unroll
      for (int j = 0; j < D; j++) a += rc[L::row(L::LO, D, i, j)] * Ut[j];
      R b = R(0);
#pragma unroll
      for (int j = 0; j < D; j++) b += rc[L::row(L::TL, D, i, j)] * Phi[j];
      r[i] = (Pb[i] - R(0.5) * (m * a + b)) - Phi[i];
    }
    it++;
    // correction dF = H (Phi_new - Phi); converged when it is at most
    // max(tol max(m, |Phi|), 64 eps |Phi|)
    R diff = R(0), pmax = R(0);
    R dF[D];
    if constexpr (CHORD && sizeof(R) == 4) {
      float2 x = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < D; j++)
        x = __ffma2_rn(*reinterpret_cast<const float2 *>(rc + L::row(L::HM, D, 0, j)), make_float2(r[j], r[j]), x);
      dF[0] = x.x;
      dF[1] = x.y;
    }
#pragma unroll
    for (int i = 0; i < D; i++) {
      R x = r[i];
      if (CHORD) {
        if (sizeof(R) == 4 && i < 2) {
          x = dF[i];
        } else {
          x = R(0);
#pragma unroll
          for (int j = 0; j < D; j++) x += rc[L::row(L::HM, D, i, j)] * r[j];
        }
      }
      dF[i] = x;
      diff = maxnan(diff, absr(x));
      pmax = maxnan(pmax, absr(Phi[i]));
    }
#pragma unroll
    for (int i = 0; i < D; i++) Phi[i] += dF[i];
    if (diff <= maxnan(tol * maxnan(m, pmax), epsn * pmax)) {
      st.conv = true;
      break;
    }
  }
  st.iters = it;
  if (FINAL) form_np<Q, R>(d, rc, m, mdev, h2m, st.rho, itau, st.U, Phi, dp);
#pragma unroll
  for (int i = 0; i < D; i++) st.F[i] = Phi[i] * rc[L::IJ];
}

}  // namespace vlb

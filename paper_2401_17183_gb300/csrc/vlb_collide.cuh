// vlb_collide.cuh -- the local part of one time step for one cell (section 2.2):
// moments (Eqs. 14, 15, 17), the implicit inertial force F (Eq. 27, with
// deltaPi of Eq. 30 and deltaN of Eq. 31), the curvilinear equilibrium
// (Eq. 33) with U~ = U + F/(2 rho), and the BGK post-collision populations
// N' = N + Omega + deltaN (Eqs. 12, 20). Shared by the step and moments kernels.
//
// Populations enter and leave as deviations d_a = N_a - w_a n_ref from a
// uniform reference n_ref = rho_0 J_ref (n_ref = 0 gives plain populations).
// The reference is the same in every cell, so advection and bounce-back move
// deviations exactly as they move populations, while every product below
// works on small numbers: that keeps FP32 rounding relative to the deviation,
// not to N. The force is carried as Phi = J F, which keeps J out of every
// product formed once per step with the same operands.
//
// Directions come in pairs (p, pbar = p + H) with c_pbar = -c_p; every sum over
// directions below is a sum over pairs of an even part (same for p and pbar)
// and an odd part (opposite signs), with the link coefficients stored as
// M_p = K_p + K_pbar and D_p = K_p - K_pbar.
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

// Direction-independent part of one evaluation for a given Phi: the
// equilibrium of Eq. 33 as J f^eq_a = w_a m (1 + x_a), x_p = xe_p + xo_p,
// x_pbar = xe_p - xo_p (only x is formed, never 1 + x), and deltaPi of Eq. 30
// with its trace.
template <int Q, typename R>
struct EvalParts {
  static constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  R xe[H + 1], xo[H + 1];
  R dP[D][D];
  R tr;
};

// weight class of a direction: 0 rest, 1 axis, 2 diagonal
template <int Q>
__host__ __device__ constexpr int wclass(int a) {
  return a == 0 ? 0 : lat_nnz<Q>(a) == 1 ? 1 : 2;
}

// Per-cell constants of one collision.
template <int Q, typename R>
struct CollideConst {
  R m, mdev, h2m, itau;
  R dfw[3];   // -(1 - 1/(2 tau)) rho w, per weight class
  R w9J[3];   // 9 w J
  R w3J[3];   // 3 w J
  R iwm[3];   // w m / tau
  R wm[3];    // w m
  R wd[3];    // w mdev
};

template <int Q, typename R>
__device__ __forceinline__ void eval_parts(const CellCoef<Q, R> &k, const CollideConst<Q, R> &cc,
                                           const R (&U)[Lat<Q>::D], const R (&Phi)[Lat<Q>::D],
                                           EvalParts<Q, R> &ev) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  R dU[D];
#pragma unroll
  for (int i = 0; i < D; i++) dU[i] = Phi[i] * cc.h2m;
  EqParts<Q, R> e;
  eq_parts<Q, R>(k.gd, U, dU, e);
  ev.xe[0] = eq_even_dev<Q, R>(e, 0);
  ev.xo[0] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    ev.xe[p] = eq_even_dev<Q, R>(e, p);
    ev.xo[p] = eq_odd<Q, R>(e, U, p);
  }
  // deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i_a (K^j_a - L^j_a) f^eq_a   (Eq. 30):
  // K_a - L_a = K_a + K_abar = M_p, a pair contributes c_p (f_p - f_pbar) with
  // f_p - f_pbar = 2 rho w_p xo_p
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) ev.dP[i][j] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const R df = cc.dfw[wclass<Q>(p)] * ev.xo[p];
    R t[D];
#pragma unroll
    for (int j = 0; j < D; j++) t[j] = k.M[p][j] * df;
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci == 0) continue;
#pragma unroll
      for (int j = 0; j < D; j++) {
        if (ci > 0)
          ev.dP[i][j] += t[j];
        else
          ev.dP[i][j] -= t[j];
      }
    }
  }
  ev.tr = R(0);
#pragma unroll
  for (int i = 0; i < D; i++) ev.tr += ev.dP[i][i];
}

// c_p.Phi and c_p.dPi.c_p for the positive direction p of a pair
template <int Q, typename R>
__device__ __forceinline__ void pair_dots(const EvalParts<Q, R> &ev, const R (&Phi)[Lat<Q>::D], int p,
                                          R &cF, R &cPc) {
  constexpr int D = Lat<Q>::D;
  cF = R(0);
  cPc = R(0);
#pragma unroll
  for (int i = 0; i < D; i++) {
    const int ci = Lat<Q>::c(p, i);
    if (ci == 0) continue;
    if (ci > 0)
      cF += Phi[i];
    else
      cF -= Phi[i];
#pragma unroll
    for (int j = 0; j < D; j++) {
      const int cj = Lat<Q>::c(p, j);
      if (cj == 0) continue;
      if (ci * cj > 0)
        cPc += ev.dP[i][j];
      else
        cPc -= ev.dP[i][j];
    }
  }
}

// Phi_new = J F_new (Eq. 27 plus the body force) for a given Phi without
// forming N'. With
//   N'_a - w_a n_ref = (1 - 1/tau) d_a + (w_a mdev + w_a m x_a)/tau + deltaN_a
// and deltaN_p = E_p + O_p, deltaN_pbar = E_p - O_p (Eq. 31, 1/T0 = 3),
//   E_p = 3 w_p J (3 c_p.dPi.c_p - tr dPi),  O_p = 3 w_p c_p.Phi,
// the sum -1/2 sum_a K_a (N'_a - w_a n_ref) is the cell constant Pb plus
//   -1/2 sum_p [M_p (E_p + w_p m xe_p / tau) + D_p (O_p + w_p m xo_p / tau)].
template <int Q, typename R>
__device__ __forceinline__ void eval_phi(const CellCoef<Q, R> &k, const CollideConst<Q, R> &cc,
                                         const R (&U)[Lat<Q>::D], const R (&Phi)[Lat<Q>::D],
                                         const R (&Pb)[Lat<Q>::D], R (&Pn)[Lat<Q>::D]) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  EvalParts<Q, R> ev;
  eval_parts<Q, R>(k, cc, U, Phi, ev);
  R acc[D];
#pragma unroll
  for (int i = 0; i < D; i++) acc[i] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    R cF, cPc;
    pair_dots<Q, R>(ev, Phi, p, cF, cPc);
    const int wc = wclass<Q>(p);
    const R Ea = cc.w9J[wc] * cPc - cc.w3J[wc] * ev.tr + cc.iwm[wc] * ev.xe[p];
    const R Oa = (R(3) * lat_w<Q, R>(p)) * cF + cc.iwm[wc] * ev.xo[p];
#pragma unroll
    for (int i = 0; i < D; i++) acc[i] += k.M[p][i] * Ea + k.Dk[p][i] * Oa;
  }
#pragma unroll
  for (int i = 0; i < D; i++) Pn[i] = Pb[i] - R(0.5) * acc[i];
}

// N' (as deviations dp_a = N'_a - w_a n_ref) and Phi_new at the same Phi:
//   N'_a = N_a + Omega_a + deltaN_a, Omega_a = -(N_a - J f^eq_a)/tau (Eqs. 12, 20),
//   N_a - J f^eq_a = (d_a - w_a mdev) - w_a m x_a,
// the non-equilibrium part formed first, so that its rounding error is relative
// to itself and not to the much larger d_a; deltaN_p = E_p + O_p and
// deltaN_pbar = E_p - O_p as in eval_phi.
template <int Q, typename R>
__device__ __forceinline__ void eval_np(const R (&d)[Q], const CellCoef<Q, R> &k,
                                        const CollideConst<Q, R> &cc, const R (&U)[Lat<Q>::D],
                                        const R (&Phi)[Lat<Q>::D], const R (&Pb)[Lat<Q>::D],
                                        R (&dp)[Q], R (&Pn)[Lat<Q>::D]) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  EvalParts<Q, R> ev;
  eval_parts<Q, R>(k, cc, U, Phi, ev);
  R acc[D];
#pragma unroll
  for (int i = 0; i < D; i++) acc[i] = R(0);
  {
    const R neq = (d[0] - cc.wd[0]) - cc.wm[0] * ev.xe[0];
    dp[0] = d[0] - cc.itau * neq - cc.w3J[0] * ev.tr;
  }
#pragma unroll
  for (int p = 1; p <= H; p++) {
    R cF, cPc;
    pair_dots<Q, R>(ev, Phi, p, cF, cPc);
    const int wc = wclass<Q>(p);
    const R Ep = cc.w9J[wc] * cPc - cc.w3J[wc] * ev.tr;
    const R Op = (R(3) * lat_w<Q, R>(p)) * cF;
    const R neqp = (d[p] - cc.wd[wc]) - cc.wm[wc] * (ev.xe[p] + ev.xo[p]);
    const R neqm = (d[p + H] - cc.wd[wc]) - cc.wm[wc] * (ev.xe[p] - ev.xo[p]);
    dp[p] = d[p] - cc.itau * neqp + (Ep + Op);
    dp[p + H] = d[p + H] - cc.itau * neqm + (Ep - Op);
    const R Ea = Ep + cc.iwm[wc] * ev.xe[p];
    const R Oa = Op + cc.iwm[wc] * ev.xo[p];
#pragma unroll
    for (int i = 0; i < D; i++) acc[i] += k.M[p][i] * Ea + k.Dk[p][i] * Oa;
  }
#pragma unroll
  for (int i = 0; i < D; i++) Pn[i] = Pb[i] - R(0.5) * acc[i];
}

// First-order move of dp from Phi to Phi + dPhi. With U~ = U + Phi/(2m):
//   d dp_a / dPhi . dPhi = (w_a / (2 tau)) dx_a/dU~ . dPhi + 3 w_a c_a . dPhi
// where dx_a/dU~ takes the U~ U~ terms of B (even in c_a) and the g^ij U~
// terms of C (odd in c_a):
//   even: 9 (c.U~)(c.dPhi) - 3 U~.dPhi
//   odd : 9/2 [(c.g.c)(c.dPhi) - T0 (2 c.g.dPhi + tr(g) c.dPhi)]
// The terms left out (the cubic U~ U~ U~ part and deltaPi) are of order |U|^2
// and Theta^2 relative to these, so for the small last correction of the
// chord iteration this leaves an error far below the FP32 unit roundoff.
template <int Q, typename R>
__device__ __forceinline__ void extrapolate(const CellCoef<Q, R> &k, const R (&U)[Lat<Q>::D],
                                            const R (&Phi)[Lat<Q>::D], R h2m,
                                            const R (&dPhi)[Lat<Q>::D], R itau, R (&dp)[Q]) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  R Ut[D], gD[D], trg = R(D), UD = R(0);
#pragma unroll
  for (int i = 0; i < D; i++) Ut[i] = U[i] + Phi[i] * h2m;
#pragma unroll
  for (int i = 0; i < D; i++) {
    R s = dPhi[i];
#pragma unroll
    for (int j = 0; j < D; j++) s += k.gd[sym<D>(i, j)] * dPhi[j];
    gD[i] = s;  // g . dPhi
    trg += k.gd[sym<D>(i, i)];
    UD += Ut[i] * dPhi[i];
  }
  const R ht = R(0.5) * itau;
  dp[0] += ht * lat_w<Q, R>(0) * (-R(3) * UD);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    R cD = R(0), cU = R(0), cgD = R(0), cgc = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci == 0) continue;
      cD += ci > 0 ? dPhi[i] : -dPhi[i];
      cU += ci > 0 ? Ut[i] : -Ut[i];
      cgD += ci > 0 ? gD[i] : -gD[i];
      cgc += R(1);
#pragma unroll
      for (int j = 0; j < D; j++) {
        const int cj = Lat<Q>::c(p, j);
        if (cj == 0) continue;
        cgc += ci * cj > 0 ? k.gd[sym<D>(i, j)] : -k.gd[sym<D>(i, j)];
      }
    }
    const R w = lat_w<Q, R>(p);
    const R ev = ht * w * (R(9) * cU * cD - R(3) * UD);
    const R od = ht * w * R(4.5) * (cgc * cD - R(kT0) * (R(2) * cgD + trg * cD)) + R(3) * w * cD;
    dp[p] += ev + od;
    dp[p + H] += ev - od;
  }
}

// x y = p + e exactly (FMA two-product)
__device__ __forceinline__ float two_prod_err(float x, float y, float p) { return fmaf(x, y, -p); }
__device__ __forceinline__ double two_prod_err(double x, double y, double p) { return fma(x, y, -p); }

// Full local collision: solve Phi = J G(Phi / J) by a chord iteration
//   Phi <- Phi + H (J G - Phi),  H = (I - L)^-1,
// where L is the part of dG/dF that depends only on the cell geometry (it
// comes from the g^ij U~ terms of Eq. 33 and the c.F term of Eq. 31; the
// remainder is of order |U| Theta, so each chord step shrinks the error by
// about that factor). With CHORD = false, H = I (plain fixed-point iteration)
// and the start value is Phi = 0; with CHORD, the start value is m times the
// rest-state force. A correction is accepted as converged when it is at most
// max(tol max(m, |Phi|), 64 eps |Phi|): eps is the unit roundoff of R, and
// Phi is a sum of some forty rounded terms of its own size, so smaller
// corrections are rounding noise.
// With FINAL every evaluation also forms N'. When the correction of an
// evaluation is accepted, N' is moved by that correction to first order
// (extrapolate), so the returned N' belongs to the corrected Phi and no
// further evaluation is needed: a cell whose start value is already within
// the tolerance costs a single evaluation.
template <int Q, typename R, bool CHORD, bool FINAL>
__device__ __forceinline__ void collide_cell(const R (&d)[Q], const CellCoef<Q, R> &k, R nref,
                                             R tau, R tol, int max_iter, R (&dp)[Q],
                                             CollideState<Q, R> &st) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
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
  CollideConst<Q, R> cc;
  cc.mdev = mdev;
  cc.m = nref + mdev;
  // rho = sum f = sum N / J; rho U = sum c f   (Eqs. 14, 15, 17)
  st.rho = cc.m / k.J;
  const R im = R(1) / cc.m;
  cc.h2m = R(0.5) * im;
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
  cc.itau = R(1) / tau;
  // -1/2 (1 - 1/(2 tau)) times the 2 of f_p - f_pbar = 2 rho w xo
  const R cpi = -(R(1) - R(0.5) * cc.itau);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const R w = c == 0 ? lat_w<Q, R>(0) : c == 1 ? lat_w<Q, R>(1) : lat_w<Q, R>(Q == 9 ? 3 : 4);
    cc.dfw[c] = cpi * st.rho * w;
    cc.w3J[c] = R(3) * w * k.J;
    cc.w9J[c] = R(9) * w * k.J;
    cc.iwm[c] = cc.itau * w * cc.m;
    cc.wm[c] = w * cc.m;
    cc.wd[c] = w * mdev;
  }
  // constant part of J F: body force m G, 1/2 sum_a L_a N_a (L_a = -K_abar), the
  // reference part -n_ref sum_a w_a K_a of both sums of Eq. 27 (the largest term,
  // the same every step: formed without rounding error from the split KW + KWL),
  // and the parts of -1/2 sum_a K_a N'_a that do not change during the
  // iteration. Over a pair,
  //   -1/2 (K_pbar d_p + K_p d_pbar) - 1/2 (1 - 1/tau)(K_p d_p + K_pbar d_pbar)
  //     = -(2 - 1/tau)/4 M_p s_p + (1/tau)/4 D_p t_p.
  R Pb[D];
  const R am = -R(0.25) * (R(2) - cc.itau), ad = R(0.25) * cc.itau;
#pragma unroll
  for (int i = 0; i < D; i++) {
    const R pr = nref * k.Kw[i];
    const R err = two_prod_err(nref, k.Kw[i], pr) + nref * k.KwL[i];
    R s = cc.m * k.G[i] - err - R(0.5) * cc.itau * mdev * k.Kw[i];
#pragma unroll
    for (int p = 1; p <= H; p++) s += am * k.M[p][i] * sp[p] + ad * k.Dk[p][i] * tp[p];
    Pb[i] = s - pr;
  }
  R Phi[D], Pn[D];
#pragma unroll
  for (int i = 0; i < D; i++) Phi[i] = CHORD ? cc.m * k.Fr[i] : R(0);
  st.conv = false;
  int it = 0;
  // correction dF = H (Phi_new - Phi); converged when it is at most
  // max(tol max(m, |Phi|), 64 eps |Phi|)
  auto correction = [&](R(&dF)[D]) -> bool {
    R r[D];
#pragma unroll
    for (int i = 0; i < D; i++) r[i] = Pn[i] - Phi[i];
    R diff = R(0), pmax = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      R x = r[i];
      if (CHORD) {
        x = R(0);
#pragma unroll
        for (int j = 0; j < D; j++) x += k.Hm[i][j] * r[j];
      }
      dF[i] = x;
      diff = maxnan(diff, absr(x));
      pmax = maxnan(pmax, absr(Phi[i]));
    }
    return diff <= maxnan(tol * maxnan(cc.m, pmax), epsn * pmax);
  };
  if (!FINAL) {
    // F only: iteration on Phi_new
    while (it < max_iter) {
      eval_phi<Q, R>(k, cc, st.U, Phi, Pb, Pn);
      it++;
      R dF[D];
      const bool ok = correction(dF);
#pragma unroll
      for (int i = 0; i < D; i++) Phi[i] += dF[i];
      if (ok) {
        st.conv = true;
        break;
      }
    }
  } else {
    // every evaluation also forms N'; the accepted correction is applied to
    // N' by extrapolation
    while (it < max_iter) {
      eval_np<Q, R>(d, k, cc, st.U, Phi, Pb, dp, Pn);
      it++;
      R dF[D];
      const bool ok = correction(dF);
      if (ok) {
        extrapolate<Q, R>(k, st.U, Phi, cc.h2m, dF, cc.itau, dp);
#pragma unroll
        for (int i = 0; i < D; i++) Phi[i] += dF[i];
        st.conv = true;
        break;
      }
#pragma unroll
      for (int i = 0; i < D; i++) Phi[i] += dF[i];
    }
  }
  st.iters = it;
  const R iJ = R(1) / k.J;
#pragma unroll
  for (int i = 0; i < D; i++) st.F[i] = Phi[i] * iJ;
}

}  // namespace vlb

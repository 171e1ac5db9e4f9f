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
// not to N.
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

// One evaluation of the collision for a given Phi = J F. Writes the
// post-collision deviations dp and returns Phi_new = J F_new (Eq. 27 plus the
// body force) in Po.
//   m = sum N = n_ref + mdev,  rho = m / J,  U~ = U + Phi / (2 m)
//   Pc = m G - 1/2 sum_a K_abar d_a - n_ref sum_a w_a K_a
// Working with J F rather than F keeps J out of every product that is formed
// once per step with the same operands.
template <int Q, typename R>
__device__ __forceinline__ void collide_eval(const R (&d)[Q], const CellCoef<Q, R> &k,
                                             const R (&U)[Lat<Q>::D], R rho, R h2m, R m,
                                             R mdev, const R (&Phi)[Lat<Q>::D],
                                             const R (&Pc)[Lat<Q>::D], R itau, R cpi,
                                             R (&dp)[Q], R (&Po)[Lat<Q>::D]) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  R dU[D];
#pragma unroll
  for (int i = 0; i < D; i++) dU[i] = Phi[i] * h2m;
  EqParts<Q, R> e;
  eq_parts<Q, R>(k.gd, U, dU, e);

  // f^eq (Eq. 33) as J f^eq_a = w_a m (1 + x_a); pair by pair x_p = xe_p + xo_p
  // and x_pbar = xe_p - xo_p. Only x is formed, never 1 + x.
  R xe[H + 1], xo[H + 1];
  xe[0] = eq_even_dev<Q, R>(e, 0);
  xo[0] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    xe[p] = eq_even_dev<Q, R>(e, p);
    xo[p] = eq_odd<Q, R>(e, U, p);
  }

  // deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i_a (K^j_a - L^j_a) f^eq_a   (Eq. 30)
  // with K_a - L_a = K_a + K_abar; a pair contributes c_p (f_p - f_pbar), and
  // f_p - f_pbar = 2 rho w_p xo_p
  R dP[D][D];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) dP[i][j] = R(0);
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const R df = R(2) * lat_w<Q, R>(p) * xo[p];
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(p, i);
      if (ci == 0) continue;
#pragma unroll
      for (int j = 0; j < D; j++) {
        const R mm = (k.K[p][j] + k.K[p + H][j]) * df;
        if (ci > 0)
          dP[i][j] += mm;
        else
          dP[i][j] -= mm;
      }
    }
  }
  R tr = R(0);
  const R cr = cpi * rho;
#pragma unroll
  for (int i = 0; i < D; i++) {
#pragma unroll
    for (int j = 0; j < D; j++) dP[i][j] *= cr;
    tr += dP[i][i];
  }

#pragma unroll
  for (int i = 0; i < D; i++) Po[i] = Pc[i];
#pragma unroll
  for (int a = 0; a < Q; a++) {
    // deltaN_a = w_a J [c.F/T0 + (c.dPi.c/T0 - tr dPi)/T0]   (Eq. 31), 1/T0 = 3
    R cF = R(0), cPc = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const int ci = Lat<Q>::c(a, i);
      if (ci == 0) continue;
      if (ci > 0)
        cF += Phi[i];
      else
        cF -= Phi[i];
#pragma unroll
      for (int j = 0; j < D; j++) {
        const int cj = Lat<Q>::c(a, j);
        if (cj == 0) continue;
        if (ci * cj > 0)
          cPc += dP[i][j];
        else
          cPc -= dP[i][j];
      }
    }
    const R w = lat_w<Q, R>(a);
    const R dN = w * (R(3) * cF + k.J * (R(3) * (R(3) * cPc - tr)));
    // N'_a = N_a + Omega_a + deltaN_a with Omega_a = -(N_a - J f^eq_a)/tau (Eqs. 12, 20);
    // N_a - J f^eq_a = (d_a - w_a mdev) - w_a m x_a
    const int pa = a <= H ? a : a - H;
    const R xa = a == 0 ? xe[0] : (a <= H ? xe[pa] + xo[pa] : xe[pa] - xo[pa]);
    const R neq = (d[a] - w * mdev) - (w * m) * xa;
    const R dpa = d[a] - neq * itau + dN;
    dp[a] = dpa;
    // J F^i gets -1/2 sum_a K^i_a d'_a   (Eq. 27; the reference part sits in Pc)
    if (a != 0) {
#pragma unroll
      for (int i = 0; i < D; i++) Po[i] -= R(0.5) * k.K[a][i] * dpa;
    }
  }
}

// x y = p + e exactly (FMA two-product)
__device__ __forceinline__ float two_prod_err(float x, float y, float p) { return fmaf(x, y, -p); }
__device__ __forceinline__ double two_prod_err(double x, double y, double p) { return fma(x, y, -p); }

// Full local collision: solve Phi = J G(Phi / J) by a chord iteration
//   Phi <- Phi + H (J G - Phi),  H = (I - L)^-1,
// where L is the part of dG/dF that depends only on the cell geometry (it
// comes from the g^ij U~ terms of Eq. 33 and the c.F term of Eq. 31; the
// remainder is of order |U| Theta). With CHORD = false, H = I (plain
// fixed-point iteration) and the start value is Phi = 0; with CHORD, the start
// value is m times the rest-state force. The iteration stops when the
// correction is at most max(tol max(m, |Phi|), 64 eps |Phi|): eps is the unit
// roundoff of R, and Phi is a sum of some forty rounded terms of its own size,
// so corrections below a few tens of ulp are rounding noise. N' is then
// evaluated once more with the corrected Phi; the chord step leaves that Phi
// about |L| |U| times the last correction away from the fixed point, which is
// what makes N' accurate to the precision of the arithmetic. (FINAL = false
// skips that evaluation when only F is wanted.)
template <int Q, typename R, bool CHORD, bool FINAL>
__device__ __forceinline__ void collide_cell(const R (&d)[Q], const CellCoef<Q, R> &k, R nref,
                                             R tau, R tol, int max_iter, R (&dp)[Q],
                                             CollideState<Q, R> &st) {
  constexpr int D = Lat<Q>::D;
  const R epsn = sizeof(R) == 4 ? R(64.0 / 16777216.0) : R(64.0 / 9007199254740992.0);
  R mdev = R(0);
#pragma unroll
  for (int a = 0; a < Q; a++) mdev += d[a];
  const R m = nref + mdev;
  // rho = sum f = sum N / J; rho U = sum c f   (Eqs. 14, 15, 17)
  st.rho = m / k.J;
  const R im = R(1) / m;
  const R h2m = R(0.5) * im;
#pragma unroll
  for (int i = 0; i < D; i++) {
    R s = R(0);
#pragma unroll
    for (int a = 1; a < Q; a++) {
      const int ci = Lat<Q>::c(a, i);
      if (ci > 0) s += d[a];
      if (ci < 0) s -= d[a];
    }
    st.U[i] = s * im;
  }
  // constant part of J F: body force m G, 1/2 sum_a L_a N_a (L_a = -K_abar) and the
  // reference part -n_ref sum_a w_a K_a of both sums of Eq. 27. The last is the
  // largest term and is the same every step, so it is formed without rounding
  // error from the split coefficient KW + KWL.
  R Pc[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    const R p = nref * k.Kw[i];
    const R err = two_prod_err(nref, k.Kw[i], p) + nref * k.KwL[i];
    Pc[i] = m * k.G[i] - err;
  }
#pragma unroll
  for (int a = 1; a < Q; a++)
#pragma unroll
    for (int i = 0; i < D; i++) Pc[i] -= R(0.5) * k.K[lat_opp<Q>(a)][i] * d[a];
#pragma unroll
  for (int i = 0; i < D; i++) Pc[i] -= nref * k.Kw[i];
  const R itau = R(1) / tau;
  const R cpi = -R(0.5) * (R(1) - R(0.5) * itau);
  R Phi[D], Pn[D];
#pragma unroll
  for (int i = 0; i < D; i++) Phi[i] = CHORD ? m * k.Fr[i] : R(0);
  st.conv = false;
  int it = 0;
  while (it < max_iter) {
    collide_eval<Q, R>(d, k, st.U, st.rho, h2m, m, mdev, Phi, Pc, itau, cpi, dp, Pn);
    it++;
    R r[D];
#pragma unroll
    for (int i = 0; i < D; i++) r[i] = Pn[i] - Phi[i];
    R diff = R(0), pmax = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      R dF = r[i];
      if (CHORD) {
        dF = R(0);
#pragma unroll
        for (int j = 0; j < D; j++) dF += k.Hm[i][j] * r[j];
      }
      diff = maxnan(diff, absr(dF));
      pmax = maxnan(pmax, absr(Phi[i]));
      Phi[i] += dF;
    }
    if (diff <= maxnan(tol * maxnan(m, pmax), epsn * pmax)) {
      st.conv = true;
      break;
    }
  }
  st.iters = it;
  const R iJ = R(1) / k.J;
#pragma unroll
  for (int i = 0; i < D; i++) st.F[i] = Phi[i] * iJ;
  if (FINAL) collide_eval<Q, R>(d, k, st.U, st.rho, h2m, m, mdev, Phi, Pc, itau, cpi, dp, Pn);
}

}  // namespace vlb

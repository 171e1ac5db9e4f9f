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
// filled except FR, the rest state and UW, which are left zero. With itau = 1/tau,
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
// so that the map of Eq. 27 reads
//   Phi_new = Pb' - 1/2 { m [PE : U~U~ + PO2 : (U~^k)^2 U~^l + LO U~] + TL Phi },
//   Pb' = Pb - 1/2 m (CE + PO1 U).
// With U~ = U + Phi / (2m) the LO term splits into 1/2 m LO U and LO Phi / 4,
// so Phi_new = Pc - 1/2 m Q(U~) - A Phi with Pc = Pb - 1/2 m (CE + (PO1 + LO) U),
// Q = PE : U~U~ + PO2 : (U~^k)^2 U~^l and A = LO/4 + TL/2, the part of the
// map's Jacobian that stays as U -> 0. The chord step with H = (I + A)^-1,
//   Phi <- Phi + H (Phi_new - Phi) = H (Pc - 1/2 m Q(U~)),
// therefore needs only H, H PE and H PO2; the record stores PO1 + LO in
// place of PO1, H - I, and H PE, H PO2 side by side (QM). PE is taken over k <= l
// with the off-diagonal entries doubled (U~U~ is symmetric).
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
    for (int j = i; j < D; j++) rec[L::GH + sym<D>(i, j)] = 0.5 * gd[i][j];
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
  double PE[D][NS], PO2[D][D][D], PO1[D][D], LO[D][D], TL[D][D];
  for (int i = 0; i < D; i++) {
    double ce = 0.0;
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        const double pe = 1.5 * itau * Rt[i][k][l];
        ce += T0 * pe * gd[k][l];
        if (k <= l) PE[i][sym<D>(k, l)] = (k == l ? 1.0 : 2.0) * pe;
      }
    rec[L::CE + i] = ce;
    for (int l = 0; l < D; l++) {
      double s = 0.0;
      for (int p = 1; p <= H; p++) s += Ao[p][i] * c[p][l];
      PO1[i][l] = 3.0 * s;
    }
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        PO2[i][k][l] = 0.0;
        if (k == l) continue;
        double s = 0.0;
        for (int p = 1; p <= H; p++) s += Ao[p][i] * c[p][l] * (3.0 * c[p][k] * c[p][k] - 1.0);
        PO2[i][k][l] = 4.5 * s;
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
      rec[L::PO1 + i * D + j] = PO1[i][j] + lo;
    }
  double A[D][D], Hm[D][D];
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) A[i][j] = (i == j ? 1.0 : 0.0) + 0.25 * LO[i][j] + 0.5 * TL[i][j];
  inverse_small<D>(A, Hm);
  // H - I: its entries are of the size of A, so rounding them leaves the
  // product (H - I) Pc, and with it the fixed point, far more accurate than
  // rounding H itself would
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++) rec[L::row(L::HM, D, i, j)] = Hm[i][j] - (i == j ? 1.0 : 0.0);
  for (int i = 0; i < D; i++) {
    for (int s = 0; s < NS; s++) {
      double v = 0.0;
      for (int j = 0; j < D; j++) v += Hm[i][j] * PE[j][s];
      rec[L::row(L::QM, L::NQ, i, s)] = v;
    }
    for (int k = 0; k < D; k++)
      for (int l = 0; l < D; l++) {
        if (k == l) continue;
        double v = 0.0;
        for (int j = 0; j < D; j++) v += Hm[i][j] * PO2[j][k][l];
        rec[L::row(L::QM, L::NQ, i, NS + offd<D>(k, l))] = v;
      }
  }
}

// x y = p + e exactly (FMA two-product)
__device__ __forceinline__ float two_prod_err(float x, float y, float p) { return fmaf(x, y, -p); }
__device__ __forceinline__ double two_prod_err(double x, double y, double p) { return fma(x, y, -p); }

// packed FP32 helpers: both lanes the same value; a 16-byte or 8-byte record load
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// The weights times 1/T0 = 3 of the axis (a1) and diagonal (a2) directions,
// chosen so that the identities of Eq. 10 that the momentum balance of a
// collision rests on hold exactly in R, not merely to rounding:
//   first moment of the U term of f^eq and of deltaN (Eqs. 28, 32),
//     3 sum_a w_a c_a c_a = I:        2 a1 + 4 a2 = 1 (D2Q9), 2 a1 + 8 a2 = 1 (D3Q19);
//   no momentum in the third-order Hermite part of Eq. 33, whose axis terms
//   carry b1 = 4 a2 (D2Q9) or 2 a2 (D3Q19) in place of a1.
// With 1/18 and 1/36 (or 1/9 and 1/36) rounded to FP32 each identity is off
// by about 3e-8, and every collision then changes the momentum by that
// fraction of U (or of the third-order part) -- an error that grows linearly
// with the number of steps. One constant is rounded; the others follow from
// the identities, and every operation in between is exact (scaling by powers
// of two, Sterbenz).
template <int Q, typename R>
struct MomentWeights;
template <typename R>
struct MomentWeights<19, R> {
  static constexpr R a2 = R(1) / R(12);
  static constexpr R a1 = (R(1) - R(8) * a2) / R(2);
  static constexpr R b1 = R(2) * a2;
  static_assert(R(2) * a1 + R(8) * a2 == R(1), "3 sum w c c = I must hold exactly");
  static_assert(R(4) * a2 - R(2) * b1 == R(0), "the cubic Hermite part must carry no momentum");
};
template <typename R>
struct MomentWeights<9, R> {
  static constexpr R a1 = R(1) / R(3);
  static constexpr R a2 = (R(1) - R(2) * a1) / R(4);
  static constexpr R b1 = R(4) * a2;
  static_assert(R(2) * a1 + R(4) * a2 == R(1), "3 sum w c c = I must hold exactly");
  static_assert(R(8) * a2 - R(2) * b1 == R(0), "the cubic Hermite part must carry no momentum");
};

// Post-collision deviations dp_a = N'_a - w_a n_ref at a given Phi:
//   N'_a = N_a + Omega_a + deltaN_a, Omega_a = -(N_a - J f^eq_a)/tau (Eqs. 12, 20).
// The non-equilibrium part is formed first, from the arrived populations
// relative to the cell's own rest state (rho = 1, U = 0 in Eq. 33),
// N_a = J w_a (1 + x^0_a) + n_a:
//   N_a - J f^eq_a = n_a - w_a (1 + x^0_a) (m - J) - w_a m (x_a - x^0_a),
// so that every term is of the size of the flow. Formed from d_a instead, the
// metric part of the rest state (w_a x^0_a, a sizeable fraction of w_a on a
// curved mesh) would enter every product, and its FP32 rounding shows up as a
// systematic error of the relaxed stress -- a viscosity error of about 1e-5.
//
// The bracket x_a of Eq. 33 divided by 3, split over a pair into an even and
// an odd part, from B and C^kkl scaled by 3/2 (T0 = 1/3); the rest state's
// part (g^ij - delta^ij) T0 of B stays out of xe (it is in x^0):
//   xe_p / 3 = c_p.Bh.c_p - tr Bh / 3,                  Bh = (3/2) U~U~,
//   xo_p / 3 = c_p.U + sum_{k != l} C2h^kl c^l_p (3 (c^k_p)^2 - 1),   C2h = (3/2) C^kkl.
// On velocity sets with components in {-1, 0, 1} the odd part only needs,
// per axis l, T0_l = U^l - sum_{k != l} C2h^kl (an axis direction) and
// T_lk = T0_l + 3 C2h^kl (a direction with components on l and k):
//   axis e_l: xo / 3 = c^l T0_l;   diagonal: xo / 3 = c^l T_lk + c^k T_kl,
// and the even part of a diagonal is Bh_ll + Bh_kk - tr Bh / 3 + 2 c^l c^k Bh_lk.
// mn = m - J is the mass of the flow. With REST the populations come in, and
// go out, relative to the cell's own rest state already (d_a = n_a, and
// dp_a = N'_a - o_a), so the subtraction of the rest deviation drops out.
// With RREC the rest state comes from the record (RR, RW); otherwise it is
// formed here from J and Gh = (g - I)/2, x^0_p / 3 = c_p.Gh.c_p - tr Gh / 3:
//   RW_p = w_p + 3 w_p (x^0_p / 3),  RR_p = w_p (J - n_ref) + 3 w_p J (x^0_p / 3),
// and then mn = mdev - sum_a RR_a. Every term is formed relative to its own
// size, and the identity behind the final pass holds for whatever J it uses,
// as long as RR, their sum and mn use the same one.
template <int Q, typename R, bool REST, bool RREC>
__device__ __forceinline__ void form_np(const R (&d)[Q], const R *__restrict__ rc, R m, R mdev, R mn,
                                        R nref, R h2m, R rho, R itau, const R (&U)[Lat<Q>::D],
                                        const R (&Phi)[Lat<Q>::D], R (&dp)[Q]) {
  using L = CoefLayout<Q>;
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H, NS = L::NS;
  static_assert(RREC || !REST, "rest-relative storage keeps the rest state in the record");
  R gh[NS];
#pragma unroll
  for (int i = 0; i < NS; i++) gh[i] = rc[L::GH + i];
  R rwc[RREC ? 1 : H + 1], rrc[RREC ? 1 : H + 1];
  if constexpr (!RREC) {
    const R Jc = rc[L::J], Jd = Jc - nref;
    R trg = gh[sym<D>(0, 0)];
#pragma unroll
    for (int i = 1; i < D; i++) trg += gh[sym<D>(i, i)];
    const R tr3 = trg * R(1.0 / 3.0);
    R rsum = R(0);
#pragma unroll
    for (int p = 0; p <= H; p++) {
      R t;
      if (p == 0) {
        t = -tr3;
      } else {
        const int l = nz_axis<Q>(p, 0), k = nz_axis<Q>(p, 1);
        if (k < 0) {
          t = gh[sym<D>(l, l)] - tr3;
        } else {
          const int sg = Lat<Q>::c(p, l) * Lat<Q>::c(p, k);
          t = fmar(R(2 * sg), gh[sym<D>(l, k)], gh[sym<D>(l, l)] + gh[sym<D>(k, k)]) - tr3;
        }
      }
      const R w = lat_w<Q, R>(p), w3 = R(3) * w;
      rwc[p] = fmar(w3, t, w);
      rrc[p] = fmar(w3 * Jc, t, w * Jd);
      rsum += p == 0 ? rrc[p] : R(2) * rrc[p];
    }
    mn = mdev - rsum;
  }
  auto rw_at = [&](int p) -> R {
    if constexpr (RREC)
      return rc[L::RW + p];
    else
      return rwc[p];
  };
  auto rr_at = [&](int p) -> R {
    if constexpr (RREC)
      return rc[L::RR + p];
    else
      return rrc[p];
  };
  const R hh = R(0.5) * h2m;
  R Ut[D], Uh[D], U2[D], Ut2x[D], v[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    Ut[i] = fmar(Phi[i], h2m, U[i]);
    Uh[i] = R(1.5) * Ut[i];
    U2[i] = Uh[i] * Ut[i];
    Ut2x[i] = Ut[i] + Ut[i];
    v[i] = Phi[i] * hh;   // (U~ - U) / 2
  }
  // Bh = (3/2) U~ U~ (T0 = 1/3), packed symmetric
  R Bh[NS];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = i; j < D; j++) Bh[sym<D>(i, j)] = Uh[i] * Ut[j];
  R tB3 = Bh[sym<D>(0, 0)];
#pragma unroll
  for (int i = 1; i < D; i++) tB3 += Bh[sym<D>(i, i)];
  tB3 *= R(1.0 / 3.0);
  // C2h^kl = (1/2) [(gd_kk U~^l + (U~^l - U^l)) + 2 gd_kl U~^k] + (3/2) (U~^k)^2 U~^l
  R C2h[D][D], Sc[D], T0[D], T[D][D];
#pragma unroll
  for (int k = 0; k < D; k++)
#pragma unroll
    for (int l = 0; l < D; l++) {
      if (k == l) continue;
      C2h[k][l] = fmar(gh[sym<D>(k, k)], Ut[l], fmar(gh[sym<D>(k, l)], Ut2x[k], fmar(U2[k], Ut[l], v[l])));
    }
  using MW = MomentWeights<Q, R>;
  R Oax[D];   // axis pairs: a1 U^l - b1 sum_{k != l} C2h^kl
#pragma unroll
  for (int l = 0; l < D; l++) {
    Sc[l] = R(0);
#pragma unroll
    for (int k = 0; k < D; k++)
      if (k != l) Sc[l] += C2h[k][l];
    T0[l] = U[l] - Sc[l];
    Oax[l] = fmar(MW::a1, U[l], -(MW::b1 * Sc[l]));
  }
#pragma unroll
  for (int l = 0; l < D; l++)
#pragma unroll
    for (int k = 0; k < D; k++)
      if (k != l) T[l][k] = fmar(R(3), C2h[k][l], T0[l]);
  // even and odd parts per pair
  R xe[H + 1], xo[H + 1];
  xe[0] = -tB3;
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const int l = nz_axis<Q>(p, 0), k = nz_axis<Q>(p, 1);
    const int sl = Lat<Q>::c(p, l);
    if (k < 0) {
      xe[p] = Bh[sym<D>(l, l)] - tB3;
      xo[p] = sl > 0 ? T0[l] : -T0[l];
    } else {
      const int sk = Lat<Q>::c(p, k);
      const R sd = (Bh[sym<D>(l, l)] + Bh[sym<D>(k, k)]) - tB3;
      xe[p] = fmar(R(2 * sl * sk), Bh[sym<D>(l, k)], sd);
      const R a = sl > 0 ? T[l][k] : -T[l][k];
      xo[p] = sk > 0 ? a + T[k][l] : a - T[k][l];
    }
  }
  // deltaPi^ij = -1/2 (1 - 1/(2 tau)) sum_a c^i_a (K^j_a - L^j_a) f^eq_a   (Eq. 30):
  // K_a - L_a = K_a + K_abar = M_p, and a pair contributes c_p (f_p - f_pbar)
  // with f_p - f_pbar = 2 rho w_p xo_p = 6 rho w_p (xo_p / 3). The record holds
  // am M_p with am = -(2 - 1/tau)/4, and -1/2 (1 - 1/(2 tau)) 2 rho = 2 rho am.
  const R r6 = R(6) * rho;
  const R r6w1 = r6 * lat_w<Q, R>(1), r6w2 = r6 * lat_w<Q, R>(Lat<Q>::H);
  R dP[D][D];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = 0; j < D; j++) dP[i][j] = R(0);
  if constexpr (sizeof(R) == 4) {
    // columns 0 and 1 in the two lanes of packed FP32 instructions
    float2 P01[D];
#pragma unroll
    for (int i = 0; i < D; i++) P01[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 1; p <= H; p++) {
      const R df = (lat_nnz<Q>(p) == 1 ? r6w1 : r6w2) * xo[p];
      const float2 am01 = ld2(rc + L::mp(p, 0));
#pragma unroll
      for (int i = 0; i < D; i++) {
        const int ci = Lat<Q>::c(p, i);
        if (ci == 0) continue;
        const R sdf = ci > 0 ? df : -df;
        P01[i] = __ffma2_rn(am01, bcast2(sdf), P01[i]);
        if constexpr (D == 3) dP[i][2] = fmar(rc[L::mp(p, 2)], sdf, dP[i][2]);
      }
    }
#pragma unroll
    for (int i = 0; i < D; i++) {
      dP[i][0] = P01[i].x;
      dP[i][1] = P01[i].y;
    }
  } else {
#pragma unroll
    for (int p = 1; p <= H; p++) {
      const R df = (lat_nnz<Q>(p) == 1 ? r6w1 : r6w2) * xo[p];
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
  }
  R tr = dP[0][0];
#pragma unroll
  for (int i = 1; i < D; i++) tr += dP[i][i];
  const R J = rc[L::J];
  // E_p = 9 w J c.dP.c - 3 w J tr dP; O_p = 3 w c.Phi (Eq. 31, 1/T0 = 3)
  const R a9_1 = (R(9) * lat_w<Q, R>(1)) * J, a9_2 = (R(9) * lat_w<Q, R>(Lat<Q>::H)) * J;
  const R tr3 = tr * R(1.0 / 3.0);
  const R b3_1 = a9_1 * tr3, b3_2 = a9_2 * tr3;
  {
    const R w = lat_w<Q, R>(0);
    const R n0 = REST ? d[0] : d[0] - rr_at(0);
    const R neq = (n0 - rw_at(0) * mn) - (R(3) * w * m) * xe[0];
    dp[0] = d[0] - itau * neq - (R(3) * w * J) * tr;
  }
  const R wm1 = MW::a1 * m, wm2 = MW::a2 * m;
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const int l = nz_axis<Q>(p, 0), k = nz_axis<Q>(p, 1);
    const int sl = Lat<Q>::c(p, l);
    const bool axis = k < 0;
    R cPc, cF;
    if (axis) {
      cPc = dP[l][l];
      cF = sl > 0 ? Phi[l] : -Phi[l];
    } else {
      const int sk = Lat<Q>::c(p, k);
      const R so = dP[l][k] + dP[k][l];
      const R sd = dP[l][l] + dP[k][k];
      cPc = sl * sk > 0 ? sd + so : sd - so;
      const R f = sl > 0 ? Phi[l] : -Phi[l];
      cF = sk > 0 ? f + Phi[k] : f - Phi[k];
    }
    const R Ep = fmar(axis ? a9_1 : a9_2, cPc, -(axis ? b3_1 : b3_2));
    const R Op = (axis ? MW::a1 : MW::a2) * cF;
    const R wm = axis ? wm1 : wm2;
    const R rw = rw_at(p);
    // odd part of J f^eq over 3 w: m xo on diagonals, m O on axis pairs
    if constexpr (sizeof(R) == 4) {
      // the pair in the two lanes of packed FP32 instructions (same roundings)
      const float2 dd = make_float2(d[p], d[p + H]);
      const float2 bs = __ffma2_rn(bcast2(-rw), bcast2(mn), REST ? dd : __fadd2_rn(dd, bcast2(-rr_at(p))));
      float2 nq;
      if (axis) {
        const R o = sl > 0 ? Oax[l] : -Oax[l];
        nq = __ffma2_rn(bcast2(-wm), bcast2(xe[p]), bs);
        nq = __ffma2_rn(make_float2(-m, m), bcast2(o), nq);
      } else {
        const float2 xs = __fadd2_rn(bcast2(xe[p]), make_float2(xo[p], -xo[p]));
        nq = __ffma2_rn(bcast2(-wm), xs, bs);
      }
      const float2 r = __fadd2_rn(__ffma2_rn(bcast2(-itau), nq, dd),
                                  __fadd2_rn(bcast2(Ep), make_float2(Op, -Op)));
      dp[p] = r.x;
      dp[p + H] = r.y;
    } else {
      R neqp, neqm;
      const R r0 = REST ? R(0) : rr_at(p);
      const R bp = fmar(-rw, mn, d[p] - r0), bm = fmar(-rw, mn, d[p + H] - r0);
      if (axis) {
        const R o = sl > 0 ? Oax[l] : -Oax[l];
        neqp = fmar(-m, o, fmar(-wm, xe[p], bp));
        neqm = fmar(m, o, fmar(-wm, xe[p], bm));
      } else {
        neqp = bp - wm * (xe[p] + xo[p]);
        neqm = bm - wm * (xe[p] - xo[p]);
      }
      dp[p] = d[p] - itau * neqp + (Ep + Op);
      dp[p + H] = d[p + H] - itau * neqm + (Ep - Op);
    }
  }
}

// Full local collision: solve the fixed point Phi = J G(Phi / J) of Eq. 27 by
// the chord iteration Phi <- H (Pc - 1/2 m Q(U~)) (see build_record), from the
// start value m times the rest-state force. A step is accepted as converged
// when its change is at most max(tol max(m, |Phi|), 64 eps |Phi|): eps is the
// unit roundoff of R, and Phi is a sum of dozens of rounded terms of its own
// size, so smaller changes are rounding noise. With FINAL, the post-collision
// deviations are formed at the converged Phi.
// rc points at the cell's coefficient record (global, shared or local
// memory); itau = 1/tau. With REST, d holds e_a = N_a - o_a relative to the
// cell's own rest state (16-bit storage, see CoefLayout), and so does dp.
template <int Q, typename R, bool FINAL, bool REST = false, bool RREC = true>
__device__ __forceinline__ void collide_cell(const R (&d)[Q], const R *__restrict__ rc, R nref,
                                             R itau, R tol, int max_iter, R (&dp)[Q],
                                             CollideState<Q, R> &st) {
  using L = CoefLayout<Q>;
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H, NS = L::NS, NQ = L::NQ;
  static_assert(D == 2 || NQ % 4 == 0, "row 2 of the chord step is read in 16-byte quads");
  const R epsn = sizeof(R) == 4 ? R(64.0 / 16777216.0) : R(64.0 / 9007199254740992.0);
  // pair sums s_p = d_p + d_pbar and differences t_p = d_p - d_pbar
  // (with REST: of e_a; the rest state's part of the s_p enters through SR)
  R sp[H + 1], tp[H + 1];
  R mdev = d[0];
#pragma unroll
  for (int p = 1; p <= H; p++) {
    sp[p] = d[p] + d[p + H];
    tp[p] = d[p] - d[p + H];
    mdev += sp[p];
  }
  // m - J, the mass of the flow
  R mn;
  if constexpr (REST) {
    mn = mdev + rc[L::MNV];
    mdev += rc[L::MDV];
  } else {
    mn = RREC ? mdev - rc[L::RR + H + 1] : R(0);   // else formed in form_np
  }
  const R m = nref + mdev;
  // rho = sum f = sum N / J; rho U = sum c f   (Eqs. 14, 15, 17)
  st.rho = m * rc[L::IJ];
  const R im = R(1) / m;
  const R h2m = R(0.5) * im;
  const R hm = R(0.5) * m;
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
  R s[D], pr[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    const R kw = rc[L::KW + i];
    pr[i] = nref * kw;
    const R err = two_prod_err(nref, kw, pr[i]) + nref * rc[L::KWL + i];
    s[i] = m * rc[L::BODY + i] - err - R(0.5) * itau * mdev * kw;
    if constexpr (REST) s[i] += rc[L::SR + i];
  }
  if constexpr (sizeof(R) == 4) {
    // components 0 and 1 in the two lanes of packed FP32 instructions, two
    // partial sums each
    float2 sa = make_float2(s[0], s[1]), sb = make_float2(0.f, 0.f);
    float s2a = D == 3 ? s[D - 1] : 0.f, s2b = 0.f;
#pragma unroll
    for (int p = 1; p <= H; p++) {
      const float4 q = ld4(rc + L::mp(p, 0));   // am M^0, am M^1, ad D^0, ad D^1
      float2 &acc = (p & 1) ? sa : sb;
      acc = __ffma2_rn(make_float2(q.x, q.y), bcast2(sp[p]), acc);
      acc = __ffma2_rn(make_float2(q.z, q.w), bcast2(tp[p]), acc);
      if constexpr (D == 3) {
        const float2 r2 = ld2(rc + L::mp(p, 2));   // am M^2, ad D^2
        float &a2 = (p & 1) ? s2a : s2b;
        a2 = fmaf(r2.x, sp[p], a2);
        a2 = fmaf(r2.y, tp[p], a2);
      }
    }
    const float2 st01 = __fadd2_rn(sa, sb);
    s[0] = st01.x;
    s[1] = st01.y;
    if constexpr (D == 3) s[D - 1] = s2a + s2b;
  } else {
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
      for (int p = 1; p <= H; p++) s[i] = fmar(rc[L::dk(p, i)], tp[p], fmar(rc[L::mp(p, i)], sp[p], s[i]));
  }
  // Pc = Pb - 1/2 m (CE + (PO1 + LO) U), then Pt = H Pc = Pc + (H - I) Pc
  R Pc[D];
#pragma unroll
  for (int i = 0; i < D; i++) {
    R u = rc[L::CE + i];
#pragma unroll
    for (int l = 0; l < D; l++) u = fmar(rc[L::PO1 + i * D + l], st.U[l], u);
    Pc[i] = (s[i] - hm * u) - pr[i];
  }
  R Pt[D];
  if constexpr (sizeof(R) == 4) {
    float2 x = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < D; j++) x = __ffma2_rn(ld2(rc + L::row(L::HM, D, 0, j)), bcast2(Pc[j]), x);
    const float2 p01 = __fadd2_rn(make_float2(Pc[0], Pc[1]), x);
    Pt[0] = p01.x;
    Pt[1] = p01.y;
    if constexpr (D == 3) {
      R y = R(0);
#pragma unroll
      for (int j = 0; j < D; j++) y = fmar(rc[L::row(L::HM, D, 2, j)], Pc[j], y);
      Pt[D - 1] = Pc[D - 1] + y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; i++) {
      R y = R(0);
#pragma unroll
      for (int j = 0; j < D; j++) y = fmar(rc[L::row(L::HM, D, i, j)], Pc[j], y);
      Pt[i] = Pc[i] + y;
    }
  }
  R Phi[D];
#pragma unroll
  for (int i = 0; i < D; i++) Phi[i] = m * rc[L::FR + i];
  st.conv = false;
  int it = 0;
  while (it < max_iter) {
    // Phi_new = H Pc - 1/2 m [H PE : U~U~ + H PO2 : (U~^k)^2 U~^l]
    R Ut[D], sq[D], mono[NQ];
#pragma unroll
    for (int i = 0; i < D; i++) {
      Ut[i] = fmar(Phi[i], h2m, st.U[i]);
      sq[i] = Ut[i] * Ut[i];
    }
#pragma unroll
    for (int k = 0; k < D; k++)
#pragma unroll
      for (int l = k; l < D; l++) mono[sym<D>(k, l)] = k == l ? sq[k] : Ut[k] * Ut[l];
#pragma unroll
    for (int k = 0; k < D; k++)
#pragma unroll
      for (int l = 0; l < D; l++)
        if (k != l) mono[NS + offd<D>(k, l)] = sq[k] * Ut[l];
    R a[D];
    if constexpr (sizeof(R) == 4) {
      // rows 0 and 1 in the two lanes of packed FP32 instructions, two partial
      // sums per row
      float2 a01a = make_float2(0.f, 0.f), a01b = make_float2(0.f, 0.f);
      float a2a = 0.f, a2b = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < NQ; s2 += 2) {
        if (s2 + 1 < NQ) {
          const float4 q = ld4(rc + L::QM + 2 * s2);
          a01a = __ffma2_rn(make_float2(q.x, q.y), bcast2(mono[s2]), a01a);
          a01b = __ffma2_rn(make_float2(q.z, q.w), bcast2(mono[s2 + 1]), a01b);
        } else {
          a01a = __ffma2_rn(ld2(rc + L::QM + 2 * s2), bcast2(mono[s2]), a01a);
        }
      }
      if constexpr (D == 3) {
#pragma unroll
        for (int s4 = 0; s4 < NQ; s4 += 4) {
          const float4 q = ld4(rc + L::row(L::QM, NQ, 2, s4));
          a2a = fmaf(q.x, mono[s4], a2a);
          a2b = fmaf(q.y, mono[s4 + 1], a2b);
          a2a = fmaf(q.z, mono[s4 + 2], a2a);
          a2b = fmaf(q.w, mono[s4 + 3], a2b);
        }
      }
      const float2 a01 = __fadd2_rn(a01a, a01b);
      a[0] = a01.x;
      a[1] = a01.y;
      if constexpr (D == 3) a[D - 1] = a2a + a2b;
    } else {
#pragma unroll
      for (int i = 0; i < D; i++) {
        R x = R(0);
#pragma unroll
        for (int s2 = 0; s2 < NQ; s2++) x = fmar(rc[L::row(L::QM, NQ, i, s2)], mono[s2], x);
        a[i] = x;
      }
    }
    it++;
    // converged when the change is at most max(tol max(m, |Phi|), 64 eps |Phi|)
    R diff = R(0), pmax = R(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const R pn = fmar(-hm, a[i], Pt[i]);
      diff = maxnan(diff, absr(pn - Phi[i]));
      pmax = maxnan(pmax, absr(Phi[i]));
      Phi[i] = pn;
    }
    if (diff <= maxnan(tol * maxnan(m, pmax), epsn * pmax)) {
      st.conv = true;
      break;
    }
  }
  st.iters = it;
  if (FINAL) form_np<Q, R, REST, RREC>(d, rc, m, mdev, mn, nref, h2m, st.rho, itau, st.U, Phi, dp);
#pragma unroll
  for (int i = 0; i < D; i++) st.F[i] = Phi[i] * rc[L::IJ];
}

}  // namespace vlb

// vlb_step.cu -- the fused stream-and-collide time step (Eq. 12 with the
// one-to-one advection of Eq. 22), one thread per cell, in place with the A-A
// access pattern over a structure-of-arrays population layout f[a][cell]:
//
//   even step: read N_a(q) from slot a of q; collide; write N'_a(q) to slot
//              abar of q (no neighbour access at all).
//   odd step : the population arriving at q along c_a is N'_a(q - c_a), which
//              the previous even step left in slot abar of q - c_a; collide;
//              write N'_a(q) to slot a of q + c_a, where the next even step
//              reads it as N_a(q + c_a).
//
// Each odd-step thread writes exactly the locations it read, so no two threads
// touch the same word. Walls (index-space halfway bounce-back) fold into the
// same addressing: a population that would leave through a wall is written to
// the cell's own slot that the next step reads as the reflected arrival.
#include "vlb_addr.cuh"
#include "vlb_collide.cuh"

namespace vlb {

struct StepArgs {
  void *f;
  const void *coef;
  int *err;
  Grid g;
  int64_t ncell;
  int64_t cstride;  // records in the coefficient array
  int64_t nfast;    // plane mode: record = cell / nfast
  double tau, tol;
  double nref;      // populations are stored as N_a - w_a nref
  int32_t max_iter;
  int32_t moving;
};

template <int Q, typename S, typename R, bool ODD, bool PLANE>
__global__ void __launch_bounds__(128) k_step(const StepArgs a) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  using L = CoefLayout<Q>;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.ncell) return;
  S *f = static_cast<S *>(a.f);
  const R *coef = static_cast<const R *>(a.coef);
  const int64_t ps = a.ncell;
  const Addr<Q> ad(a.g, cell);

  // ---- pull (read side of Eq. 22): deviations d_a = N_a - w_a n_ref
  R N[Q];
  pull<Q, ODD, S, R>(f, ps, ad, N);

  // ---- coefficients
  const int64_t rec = PLANE ? cell / a.nfast : cell;
  const int64_t cs = a.cstride;
  CellCoef<Q, R> k;
  k.J = coef[L::J * cs + rec];
#pragma unroll
  for (int i = 0; i < L::NS; i++) k.gd[i] = coef[(L::GINV + i) * cs + rec];
#pragma unroll
  for (int i = 0; i < D; i++) {
    k.G[i] = coef[(L::BODY + i) * cs + rec];
    k.Kw[i] = coef[(L::KW + i) * cs + rec];
    k.KwL[i] = coef[(L::KWL + i) * cs + rec];
    k.Fr[i] = coef[(L::FR + i) * cs + rec];
    k.K[0][i] = R(0);
#pragma unroll
    for (int j = 0; j < D; j++) k.Hm[i][j] = coef[(L::HM + i * D + j) * cs + rec];
  }
#pragma unroll
  for (int av = 1; av < Q; av++)
#pragma unroll
    for (int i = 0; i < D; i++) k.K[av][i] = coef[(L::K + (av - 1) * D + i) * cs + rec];

  // ---- collide (section 2.2)
  R Np[Q];
  CollideState<Q, R> cst;
  collide_cell<Q, R, true, true>(N, k, R(a.nref), R(a.tau), R(a.tol), a.max_iter, Np,
                                           cst);
  if (!cst.conv) atomicOr(a.err, ERR_NOCONV);

  // ---- moving walls: a reflected population is corrected by
  //      -J rho [f^eq_a - f^eq_abar](rho = 1, U = U~ = U_wall)
  const bool moving = a.moving && ad.wall_cell();
  R uw[D];
#pragma unroll
  for (int i = 0; i < D; i++) uw[i] = moving ? coef[(L::UW + i) * cs + rec] : R(0);
  EqParts<Q, R> ew;
  if (moving) {
    R zero[D];
#pragma unroll
    for (int i = 0; i < D; i++) zero[i] = R(0);
    eq_parts<Q, R>(k.gd, uw, zero, ew);
  }

  // ---- push (write side of Eq. 22)
#pragma unroll
  for (int av = 1; av < Q; av++) {
    const int ab = lat_opp<Q>(av);
    const bool cr = ad.crosses(av, 1);
    R v = Np[av];
    if (moving && cr) {
      const int p = av <= H ? av : av - H;
      const R O = eq_odd<Q, R>(ew, uw, p);
      const R corr = R(2) * k.J * cst.rho * lat_w<Q, R>(av) * O;
      v -= (av <= H) ? corr : -corr;
    }
    if (!ODD || cr)
      f[ab * ps + cell] = static_cast<S>(v);
    else
      f[av * ps + ad.nb(av, 1)] = static_cast<S>(v);
  }
  f[cell] = static_cast<S>(Np[0]);
}

template <int Q, typename S, typename R>
static cudaError_t launch_step_t(const vlb_sim *sim, int odd, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  StepArgs a;
  a.f = sim->d_f;
  a.coef = sim->d_coef;
  a.err = sim->d_err;
  a.g = make_grid(m);
  a.ncell = m->ncell;
  a.cstride = sim->ncoef;
  a.nfast = m->md.n[m->md.dim - 1];
  a.tau = sim->p.tau;
  a.tol = sim->p.tol;
  a.nref = sim->nref;
  a.max_iter = sim->p.max_iter;
  a.moving = 0;
  for (int ax = 0; ax < 3; ax++)
    for (int sd = 0; sd < 2; sd++)
      for (int d = 0; d < 3; d++)
        if (sim->p.wall_u[ax][sd][d] != 0.0 || sim->p.wall_omega[ax][sd][d] != 0.0) a.moving = 1;
  const int threads = 128;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  if (sim->plane) {
    if (odd)
      k_step<Q, S, R, true, true><<<(unsigned)blocks, threads, 0, s>>>(a);
    else
      k_step<Q, S, R, false, true><<<(unsigned)blocks, threads, 0, s>>>(a);
  } else {
    if (odd)
      k_step<Q, S, R, true, false><<<(unsigned)blocks, threads, 0, s>>>(a);
    else
      k_step<Q, S, R, false, false><<<(unsigned)blocks, threads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const vlb_sim *sim, int odd, cudaStream_t s) {
  const int q = sim->mesh->md.q;
  const bool f64 = sim->p.precision == VLB_F64;
  if (q == 9) {
    return f64 ? launch_step_t<9, double, double>(sim, odd, s)
               : launch_step_t<9, float, float>(sim, odd, s);
  }
  return f64 ? launch_step_t<19, double, double>(sim, odd, s)
             : launch_step_t<19, float, float>(sim, odd, s);
}

}  // namespace vlb

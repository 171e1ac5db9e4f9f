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
  int32_t plane;    // one coefficient record per column of the fastest axis
  double tau, tol;
  double nref;      // populations are stored as N_a - w_a nref
  int32_t max_iter;
  int32_t moving;
};

// One thread per cell. The grid is (tiles of the fastest axis, the middle
// axis, the slowest axis), so a thread finds its cell without a division and
// the 32 cells of a warp share every other coordinate: wall tests are
// warp-uniform and, in plane mode, so is the coefficient record. IT is the
// index type: 32-bit whenever q * ncell fits.
constexpr int kStepThreads = 128;

// read RS values of type R from a 16-byte aligned record with vector loads
// through the read-only path
template <typename R, int RS>
__device__ __forceinline__ void load_record(const R *__restrict__ p, R (&out)[RS]) {
  if constexpr (sizeof(R) == 4) {
    static_assert(RS % 4 == 0, "record stride must be a multiple of 16 bytes");
    const float4 *v = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < RS / 4; i++) {
      const float4 x = __ldg(v + i);
      out[4 * i] = x.x;
      out[4 * i + 1] = x.y;
      out[4 * i + 2] = x.z;
      out[4 * i + 3] = x.w;
    }
  } else {
    static_assert(RS % 2 == 0, "record stride must be a multiple of 16 bytes");
    const double2 *v = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < RS / 2; i++) {
      const double2 x = __ldg(v + i);
      out[2 * i] = x.x;
      out[2 * i + 1] = x.y;
    }
  }
}

template <int Q, typename S, typename R, bool ODD, typename IT>
__global__ void __launch_bounds__(kStepThreads, sizeof(R) == 4 ? 3 : 1) k_step(const StepArgs a) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  using L = CoefLayout<Q>;
  const IT ifast = (IT)blockIdx.x * kStepThreads + (IT)threadIdx.x;
  const IT nfast = (IT)(D == 3 ? a.g.n[2] : a.g.n[1]);
  if (ifast >= nfast) return;
  const Addr<Q, IT> ad = D == 3 ? Addr<Q, IT>(a.g, (IT)blockIdx.z, (IT)blockIdx.y, ifast)
                                : Addr<Q, IT>(a.g, (IT)blockIdx.y, ifast, (IT)0);
  const IT cell = ad.cell;
  S *__restrict__ f = static_cast<S *>(a.f);
  const R *__restrict__ coef = static_cast<const R *>(a.coef);
  const IT ps = (IT)a.ncell;

  // ---- pull (read side of Eq. 22): deviations d_a = N_a - w_a n_ref
  R N[Q];
  pull<Q, ODD, S, R, IT>(f, ps, ad, N);

  // ---- coefficients: one record per column of the fastest axis (plane mode)
  // or per cell, read with 16-byte vector loads
  const IT rec = a.plane ? (D == 3 ? (IT)blockIdx.z * (IT)a.g.n[1] + (IT)blockIdx.y : (IT)blockIdx.y)
                         : cell;
  constexpr int RS = L::template stride<R>();
  R rv[RS];
  load_record<R, RS>(coef + (int64_t)rec * RS, rv);
  CellCoef<Q, R> k;
  k.J = rv[L::J];
#pragma unroll
  for (int i = 0; i < L::NS; i++) k.gd[i] = rv[L::GINV + i];
#pragma unroll
  for (int i = 0; i < D; i++) {
    k.G[i] = rv[L::BODY + i];
    k.Kw[i] = rv[L::KW + i];
    k.KwL[i] = rv[L::KWL + i];
    k.Fr[i] = rv[L::FR + i];
    k.M[0][i] = k.Dk[0][i] = R(0);
#pragma unroll
    for (int j = 0; j < D; j++) k.Hm[i][j] = rv[L::HM + i * D + j];
  }
#pragma unroll
  for (int p = 1; p <= H; p++)
#pragma unroll
    for (int i = 0; i < D; i++) {
      k.M[p][i] = rv[L::MP + (p - 1) * D + i];
      k.Dk[p][i] = rv[L::DK + (p - 1) * D + i];
    }

  // ---- collide (section 2.2)
  R Np[Q];
  CollideState<Q, R> cst;
  collide_cell<Q, R, true, true>(N, k, R(a.nref), R(a.tau), R(a.tol), a.max_iter, Np, cst);
  if (!cst.conv) atomicOr(a.err, ERR_NOCONV);

  // ---- moving walls: a reflected population is corrected by
  //      -J rho [f^eq_a - f^eq_abar](rho = 1, U = U~ = U_wall)
  const bool moving = a.moving && ad.wall_cell();
  R uw[D];
#pragma unroll
  for (int i = 0; i < D; i++) uw[i] = moving ? rv[L::UW + i] : R(0);
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
    const bool crs = ad.crosses(av, 1);
    R v = Np[av];
    if (moving && crs) {
      const int p = av <= H ? av : av - H;
      const R O = eq_odd<Q, R>(ew, uw, p);
      const R corr = R(2) * k.J * cst.rho * lat_w<Q, R>(av) * O;
      v -= (av <= H) ? corr : -corr;
    }
    if (!ODD || crs)
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
  a.plane = sim->plane;
  a.tau = sim->p.tau;
  a.tol = sim->p.tol;
  a.nref = sim->nref;
  a.max_iter = sim->p.max_iter;
  a.moving = 0;
  for (int ax = 0; ax < 3; ax++)
    for (int sd = 0; sd < 2; sd++)
      for (int d = 0; d < 3; d++)
        if (sim->p.wall_u[ax][sd][d] != 0.0 || sim->p.wall_omega[ax][sd][d] != 0.0) a.moving = 1;
  const int dim = m->md.dim;
  const int64_t nfast = dim == 3 ? m->md.n[2] : m->md.n[1];
  dim3 grid((unsigned)((nfast + kStepThreads - 1) / kStepThreads),
            (unsigned)(dim == 3 ? m->md.n[1] : m->md.n[0]), (unsigned)(dim == 3 ? m->md.n[0] : 1));
  // 32-bit indexing when every population offset fits
  const bool i32 = (int64_t)Q * m->ncell < ((int64_t)1 << 31);
  if (i32) {
    if (odd)
      k_step<Q, S, R, true, int32_t><<<grid, kStepThreads, 0, s>>>(a);
    else
      k_step<Q, S, R, false, int32_t><<<grid, kStepThreads, 0, s>>>(a);
  } else {
    if (odd)
      k_step<Q, S, R, true, int64_t><<<grid, kStepThreads, 0, s>>>(a);
    else
      k_step<Q, S, R, false, int64_t><<<grid, kStepThreads, 0, s>>>(a);
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

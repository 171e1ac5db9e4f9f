// vlb_moments.cu -- output mapping of Eq. 34 (rho, u = U^i g_i and
// u~ = U~^i g_i), FP64 conservation sums (mass, P = sum e_a N_a and the
// invariant M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a) reduced with warp
// shuffles, and the population gather/scatter used for checkpoints.
#include "vlb_addr.cuh"
#include "vlb_collide.cuh"

namespace vlb {

struct MomArgs {
  const void *f;
  Grid g;
  int64_t ncell;
  const double *gl;
  // the simulation's coefficient records (FP64 or FP32; one per cell, or one
  // per column of the fastest axis in plane mode)
  const void *coef;
  int32_t plane;
  double nref, tol;
  int64_t nfast;
  int64_t rs;
  double rot[3][9];
  int32_t has_rot[3];
  int32_t periodic[3];
  double tau;
  RefCtx ref;
  int *err;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block sum of NV values into out[0..NV) (thread 0 writes)
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *out) {
  __shared__ double sh[NV][kMomThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[k] = s;
    }
  }
}

// MT: arithmetic of the per-cell solve for F -- FP64 for FP64 simulations,
// FP32 (the step kernel's own arithmetic, on deviations from n_ref) for the
// others; the output mapping and the conservation sums are FP64 throughout.
template <int Q, typename S, bool ODD, typename MT>
__global__ void __launch_bounds__(kMomThreads) k_moments(const MomArgs a, double *out,
                                                         double *partial) {
  constexpr int D = Lat<Q>::D;
  const S *f = static_cast<const S *>(a.f);
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const Addr<Q> ad(a.g, c);
    double N[Q];
    pull_abs<Q, ODD, S>(f, a.ncell, ad, a.ref, N);
    // the cell's coefficient record (stored in MT) and its deviations from
    // the uniform reference
    const MT *rec = static_cast<const MT *>(a.coef) + (a.plane ? c / a.nfast : c) * a.rs;
    MT dv[Q];
#pragma unroll
    for (int av = 0; av < Q; av++) dv[av] = static_cast<MT>(N[av] - lat_w<Q, double>(av) * a.nref);
    MT Np[Q];
    CollideState<Q, MT> st;
    // chord iteration from the record's rest-state start value
    collide_cell<Q, MT, false>(dv, rec, static_cast<MT>(a.nref), static_cast<MT>(1.0 / a.tau),
                                     static_cast<MT>(a.tol), 200, Np, st);
    if (!st.conv) atomicOr(a.err, ERR_NOCONV);
    double gl[D][D];
    for (int i = 0; i < D; i++)
      for (int d = 0; d < D; d++) gl[i][d] = a.gl[(c * D + i) * D + d];
    // fields as three arrays: rho [ncell], u [ncell][D], u~ [ncell][D]
    double *o_u = out + a.ncell + c * D, *o_ut = out + a.ncell * (1 + D) + c * D;
    const double rho = st.rho;
    out[c] = rho;
    bool finite = isfinite(rho);
    for (int d = 0; d < D; d++) {
      double uu = 0.0, ut = 0.0;
      for (int i = 0; i < D; i++) {
        const double Ui = st.U[i], Fi = st.F[i];
        uu += Ui * gl[i][d];                                        // u = U^i g_i (Eq. 34)
        ut += (Ui + 0.5 * (Fi / rho)) * gl[i][d];                   // u~ = U~^i g_i
      }
      o_u[d] = uu;
      o_ut[d] = ut;
      finite = finite && isfinite(uu) && isfinite(ut);
    }
    if (!finite) atomicOr(a.err, ERR_NONFINITE);
    // conservation sums
#pragma unroll 1
    for (int av = 0; av < Q; av++) {
      acc[0] += N[av];
      double e[D], eb[D];
      for (int d = 0; d < D; d++) {
        double s = 0.0;
        for (int i = 0; i < D; i++) s += Lat<Q>::c(av, i) * gl[i][d];
        e[d] = s;
        eb[d] = s;
      }
      if (av != 0 && !ad.crosses(av, -1)) {
        // e_a at q - c_a: tangents of the wrapped neighbour, rotated back if the
        // step crosses a periodic seam that carries a rotation
        const int64_t nb = ad.nb(av, -1);
        double gn[D][D];
        for (int i = 0; i < D; i++)
          for (int d = 0; d < D; d++) gn[i][d] = a.gl[(nb * D + i) * D + d];
        for (int ax = 0; ax < D; ax++) {
          const int cax = Lat<Q>::c(av, ax);
          if (!a.has_rot[ax] || !a.periodic[ax] || cax == 0) continue;
          const bool below = (cax > 0 && ad.ic[ax] == 0);             // image at index -1: R^T
          const bool above = (cax < 0 && ad.ic[ax] == a.g.n[ax] - 1);  // image at index n: R
          if (!below && !above) continue;
          const double *R = a.rot[ax];
          for (int i = 0; i < D; i++) {
            double y[D];
            for (int r = 0; r < D; r++) {
              double s = 0.0;
              for (int cc = 0; cc < D; cc++) s += (above ? R[3 * r + cc] : R[3 * cc + r]) * gn[i][cc];
              y[r] = s;
            }
            for (int r = 0; r < D; r++) gn[i][r] = y[r];
          }
        }
        for (int d = 0; d < D; d++) {
          double s = 0.0;
          for (int i = 0; i < D; i++) s += Lat<Q>::c(av, i) * gn[i][d];
          eb[d] = s;
        }
      }
      for (int d = 0; d < D; d++) {
        acc[1 + d] += e[d] * N[av];
        acc[4 + d] += 0.5 * (e[d] + eb[d]) * N[av];
      }
    }
  }
  block_sum<7>(acc, partial + (int64_t)blockIdx.x * 7);
}

template <int Q, typename S>
static cudaError_t moments_t(const vlb_sim *sim, double *d_out, double *d_partial, int64_t nblk,
                             cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  MomArgs a;
  a.f = sim->d_f;
  a.g = make_grid(m);
  a.ncell = m->ncell;
  a.gl = m->d_gl;
  a.coef = sim->d_coef;
  a.nref = sim->nref;
  a.tol = sim->p.tol;
  a.plane = sim->plane;
  a.nfast = m->md.n[m->md.dim - 1];
  a.rs = sim->nc;
  for (int d = 0; d < 3; d++) {
    a.has_rot[d] = m->md.has_rot[d];
    a.periodic[d] = (d < m->md.dim && m->md.bc[d] == VLB_PERIODIC) ? 1 : 0;
    for (int k = 0; k < 9; k++) a.rot[d][k] = m->md.rot[d][k];
  }
  a.tau = sim->p.tau;
  a.ref = make_ref(sim);
  a.err = sim->d_err;
  using MT = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
  if (sim->t & 1)
    k_moments<Q, S, true, MT><<<(unsigned)nblk, kMomThreads, 0, s>>>(a, d_out, d_partial);
  else
    k_moments<Q, S, false, MT><<<(unsigned)nblk, kMomThreads, 0, s>>>(a, d_out, d_partial);
  return cudaGetLastError();
}

cudaError_t launch_moments(const vlb_sim *sim, double *d_out, double *d_partial, int64_t nblk,
                           cudaStream_t s) {
  return with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return sim->mesh->md.q == 9 ? moments_t<9, S>(sim, d_out, d_partial, nblk, s)
                                : moments_t<19, S>(sim, d_out, d_partial, nblk, s);
  });
}

// fixed-order reduction of the per-block partial sums (deterministic)
__global__ void __launch_bounds__(kMomThreads) k_finish_totals(const double *partial, int64_t nblk,
                                                               double *totals) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int k = 0; k < 7; k++) v[k] += partial[b * 7 + k];
  block_sum<7>(v, totals);
}

cudaError_t launch_finish_totals(const double *d_partial, int64_t nblk, double *d_totals,
                                 cudaStream_t s) {
  k_finish_totals<<<1, kMomThreads, 0, s>>>(d_partial, nblk, d_totals);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ state gather / scatter
template <int Q, typename S, bool ODD>
__global__ void k_get_state(const S *f, Grid g, int64_t ncell, RefCtx ref, double *N_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const Addr<Q> ad(g, c);
  double N[Q];
  pull_abs<Q, ODD, S>(f, ncell, ad, ref, N);
#pragma unroll
  for (int a = 0; a < Q; a++) N_out[a * ncell + c] = N[a];
}

// writes the even-parity layout (slot a of q holds N_a(q))
template <int Q, typename S>
__global__ void k_set_state(S *f, int64_t ncell, RefCtx ref, const double *N_in) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
#pragma unroll
  for (int a = 0; a < Q; a++) f[a * ncell + c] = store_s<S>(N_in[a * ncell + c] - ref_at<Q>(ref, a, c));
}

cudaError_t launch_get_state(const vlb_sim *sim, double *d_N, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  const int threads = 256;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  const Grid g = make_grid(m);
  const RefCtx ref = make_ref(sim);
  return with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    const S *f = (const S *)sim->d_f;
    if (m->md.q == 9) {
      if (sim->t & 1)
        k_get_state<9, S, true><<<(unsigned)blocks, threads, 0, s>>>(f, g, m->ncell, ref, d_N);
      else
        k_get_state<9, S, false><<<(unsigned)blocks, threads, 0, s>>>(f, g, m->ncell, ref, d_N);
    } else {
      if (sim->t & 1)
        k_get_state<19, S, true><<<(unsigned)blocks, threads, 0, s>>>(f, g, m->ncell, ref, d_N);
      else
        k_get_state<19, S, false><<<(unsigned)blocks, threads, 0, s>>>(f, g, m->ncell, ref, d_N);
    }
    return cudaGetLastError();
  });
}

cudaError_t launch_set_state(const vlb_sim *sim, const double *d_N, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  const int threads = 256;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  const RefCtx ref = make_ref(sim);
  return with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    if (m->md.q == 9)
      k_set_state<9, S><<<(unsigned)blocks, threads, 0, s>>>((S *)sim->d_f, m->ncell, ref, d_N);
    else
      k_set_state<19, S><<<(unsigned)blocks, threads, 0, s>>>((S *)sim->d_f, m->ncell, ref, d_N);
    return cudaGetLastError();
  });
}

}  // namespace vlb

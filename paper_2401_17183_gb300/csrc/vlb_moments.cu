// vlb_moments.cu -- output mapping of Eq. 34 (rho, u = U^i g_i and
// u~ = U~^i g_i), FP64 conservation sums (mass, P = sum e_a N_a and the
// invariant M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a) reduced with warp
// shuffles -- shared by vlb_moments and vlb_totals_noalloc -- and the
// population gather/scatter used for checkpoints.
#include <algorithm>

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

// MT: arithmetic of the per-cell solve for F and of the output mapping --
// FP64 for FP64 simulations, FP32 (the step kernel's own arithmetic, on
// deviations from n_ref) for the others; the conservation sums are FP64
// throughout.
// One cell per thread; IT is the index type (32-bit when every population
// offset fits). In plane mode the tangents, like the coefficient record, are
// those of the column (its first cell).
template <int Q, typename S, bool ODD, typename MT, typename IT>
__global__ void __launch_bounds__(kMomThreads) k_moments(const MomArgs a, double *out) {
  constexpr int D = Lat<Q>::D;
  const S *f = static_cast<const S *>(a.f);
  const IT c = (IT)blockIdx.x * (IT)blockDim.x + (IT)threadIdx.x;
  if ((int64_t)c >= a.ncell) return;
  // index coordinates without 64-bit divisions when IT is 32-bit
  const IT n2 = (IT)a.g.n[2], n1 = (IT)a.g.n[1];
  const IT r = c / n2, i2 = c - r * n2, i0 = r / n1, i1 = r - i0 * n1;
  const Addr<Q, IT> ad(a.g, i0, i1, i2);
  // the arrived populations as deviations from the uniform reference w_a n_ref,
  // in MT: the stored value itself, plus (16-bit storage relative to the rest
  // state) the location's offset from the uniform reference
  MT dv[Q];
#pragma unroll
  for (int av = 0; av < Q; av++) {
    int slot;
    IT loc;
    arrived_loc<Q, ODD, IT>(ad, av, slot, loc);
    const S v = f[(IT)slot * (IT)a.ncell + loc];
    if constexpr (sizeof(MT) == 8) {
      dv[av] = load_s<double>(v) + (ref_at<Q>(a.ref, slot, (int64_t)loc) - lat_w<Q, double>(slot) * a.nref);
    } else {
      dv[av] = load_s<MT>(v);
      if (a.ref.rest)
        dv[av] += static_cast<MT>(ref_at<Q>(a.ref, slot, (int64_t)loc) - lat_w<Q, double>(slot) * a.nref);
    }
  }
  // the cell's (or column's) coefficient record, stored in MT
  const IT c0 = a.plane ? c - ad.ic[D - 1] : c;   // the fastest axis has stride 1
  const MT *rec = static_cast<const MT *>(a.coef) + (int64_t)(a.plane ? c0 / (IT)a.nfast : c) * a.rs;
  MT Np[Q];
  CollideState<Q, MT> st;
  // chord iteration from the record's rest-state start value
  collide_cell<Q, MT, false>(dv, rec, static_cast<MT>(a.nref), static_cast<MT>(1.0 / a.tau),
                             static_cast<MT>(a.tol), 200, Np, st);
  if (!st.conv) atomicOr(a.err, ERR_NOCONV);
  // the output mapping in the simulation's arithmetic (U and F are MT already)
  MT gl[D][D];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int d = 0; d < D; d++) gl[i][d] = static_cast<MT>(a.gl[((int64_t)c0 * D + i) * D + d]);
  // fields as three arrays: rho [ncell], u [ncell][D], u~ [ncell][D]
  double *o_u = out + a.ncell + (int64_t)c * D, *o_ut = out + a.ncell * (1 + D) + (int64_t)c * D;
  const MT rho = st.rho;
  out[c] = rho;
  bool finite = isfinite(rho);
  const MT h2r = MT(0.5) / rho;
#pragma unroll
  for (int d = 0; d < D; d++) {
    MT uu = MT(0), ut = MT(0);
#pragma unroll
    for (int i = 0; i < D; i++) {
      const MT Ui = st.U[i], Fi = st.F[i];
      uu += Ui * gl[i][d];                                        // u = U^i g_i (Eq. 34)
      ut += (Ui + Fi * h2r) * gl[i][d];                           // u~ = U~^i g_i
    }
    o_u[d] = uu;
    o_ut[d] = ut;
    finite = finite && isfinite(uu) && isfinite(ut);
  }
  if (!finite) atomicOr(a.err, ERR_NONFINITE);
}

template <int Q, typename S>
static cudaError_t moments_t(const vlb_sim *sim, double *d_out, int64_t nblk, cudaStream_t s) {
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
  const int64_t blocks = (m->ncell + kMomThreads - 1) / kMomThreads;
  const bool i32 = (int64_t)Q * m->ncell + kMomThreads < ((int64_t)1 << 31);
  const bool odd = sim->t & 1;
  if (i32) {
    if (odd)
      k_moments<Q, S, true, MT, int32_t><<<(unsigned)blocks, kMomThreads, 0, s>>>(a, d_out);
    else
      k_moments<Q, S, false, MT, int32_t><<<(unsigned)blocks, kMomThreads, 0, s>>>(a, d_out);
  } else {
    if (odd)
      k_moments<Q, S, true, MT, int64_t><<<(unsigned)blocks, kMomThreads, 0, s>>>(a, d_out);
    else
      k_moments<Q, S, false, MT, int64_t><<<(unsigned)blocks, kMomThreads, 0, s>>>(a, d_out);
  }
  (void)nblk;
  return cudaGetLastError();
}

cudaError_t launch_moments(const vlb_sim *sim, double *d_out, int64_t nblk, cudaStream_t s) {
  return with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return sim->mesh->md.q == 9 ? moments_t<9, S>(sim, d_out, nblk, s)
                                : moments_t<19, S>(sim, d_out, nblk, s);
  });
}

// ------------------------------------------------------------------ conservation totals
// mass = sum_q sum_a N_a(q), P = sum_q sum_a e_a(q) N_a(q) and the invariant
// M = sum_q sum_a 1/2 [e_a(q) + e_a(q - c_a)] N_a(q), e_a = c^i_a g_i (Eq. 9),
// with e_a(q - c_a) := e_a(q) where q - c_a lies behind a wall, and the
// tangents of a periodic image rotated by the seam's R (index n) or R^T
// (index -1). Every sum is FP64.
struct TotArgs {
  const void *f;
  Grid g;
  int64_t ncell, nfast, ncol;
  const double *gl;  // tangents g_i, [ncell][dim][dim] (component d of g_i at i * dim + d)
  RefCtx ref;
  double rot[3][9];
  int32_t has_rot[3];
  int32_t periodic[3];
};

// velocity components by a runtime direction index (constant memory)
template <int Q>
struct DirTable {
  int8_t c[Q][4];
};
template <int Q>
constexpr DirTable<Q> make_dir_table() {
  DirTable<Q> t{};
  for (int a = 0; a < Q; a++)
    for (int d = 0; d < 3; d++) t.c[a][d] = (int8_t)Lat<Q>::c(a, d);
  return t;
}
__constant__ DirTable<9> kDir9 = make_dir_table<9>();
__constant__ DirTable<19> kDir19 = make_dir_table<19>();
template <int Q>
__device__ __forceinline__ const int8_t *dir_table(int a) {
  return Q == 9 ? kDir9.c[a] : kDir19.c[a];
}

// does q - c_a leave the domain through a wall (runtime direction)
template <int Q, typename IT>
__device__ __forceinline__ bool crosses_rt(const Addr<Q, IT> &ad, const int8_t *cv) {
  bool x = false;
#pragma unroll
  for (int d = 0; d < Lat<Q>::D; d++) {
    if (cv[d] < 0) x = x || ad.hi[d];
    if (cv[d] > 0) x = x || ad.lo[d];
  }
  return x;
}

// (hi, lo) += x with the rounding error of hi + x carried in lo (TwoSum)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// N_a at a storage location, absolute (stored deviation plus its reference)
template <int Q, typename S>
__device__ __forceinline__ double loc_abs(const S *f, int64_t ncell, const RefCtx &ref, int slot,
                                          int64_t cell) {
  return load_s<double>(f[(int64_t)slot * ncell + cell]) + ref_at<Q>(ref, slot, cell);
}

// y = R x (above) or R^T x (below) for the first D components
template <int D>
__device__ __forceinline__ void rot_vec(const double *R, bool above, const double *x, double *y) {
#pragma unroll
  for (int r = 0; r < D; r++) {
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < D; c++) v += (above ? R[3 * r + c] : R[3 * c + r]) * x[c];
    y[r] = v;
  }
}

// Plane mode with a periodic fastest axis that carries no rotation: the
// tangents, hence every e_a and 1/2 [e_a(q) + e_a(q - c_a)], are constant along
// a column, so a column contributes sum_a E_a S_a with S_a the sum of N_a over
// its cells. Under the A-A layout the arrived N_a of a whole column is one
// stored row: slot a of the column (even parity, or a link from behind a
// wall) or slot abar of the column one step back along c_a (odd parity; the
// shift along the fastest axis only rotates the periodic row). A work item is
// a piece of at most kTotChunk cells of one column; one warp per item
// (grid-stride) sums the Q row pieces, then its lanes weigh them, one
// direction each.
constexpr int64_t kTotChunk = 4096;
template <int Q, typename S, bool ODD>
__global__ void __launch_bounds__(kMomThreads, 2) k_totals_plane(const TotArgs a, double *partial) {
  constexpr int D = Lat<Q>::D, NW = kMomThreads / 32;
  const S *f = static_cast<const S *>(a.f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t nchunk = (a.nfast + kTotChunk - 1) / kTotChunk;
  // one warp per work item (a piece of one column), no block barriers
  for (int64_t item = (int64_t)blockIdx.x * NW + warp; item < a.ncol * nchunk;
       item += (int64_t)gridDim.x * NW) {
    const int64_t col = item / nchunk;
    const int64_t k0 = (item - col * nchunk) * kTotChunk;
    const int64_t k1 = k0 + kTotChunk < a.nfast ? k0 + kTotChunk : a.nfast;
    // the column's first cell and its slow coordinates
    const int64_t c0 = col * a.nfast;
    const Addr<Q> ad(a.g, c0);
    // start of the stored row that holds the arrived N_a of the column
    int64_t row[Q];
#pragma unroll
    for (int av = 0; av < Q; av++) {
      if (!ODD || av == 0 || ad.crosses(av, -1)) {
        row[av] = (int64_t)av * a.ncell + c0;
      } else {
        // slot abar of the column one step back along the slow axes of c_a (the
        // fastest-axis part of the step stays in the periodic row)
        int64_t r = c0;
#pragma unroll
        for (int d = 0; d < D - 1; d++) {
          const int cd = -Lat<Q>::c(av, d);
          if (cd > 0) r += ad.dp[d];
          if (cd < 0) r += ad.dm[d];
        }
        row[av] = (int64_t)lat_opp<Q>(av) * a.ncell + r;
      }
    }
    double Sa = 0.0;
    if constexpr (sizeof(S) == 8) {
      double sum[Q];
#pragma unroll
      for (int av = 0; av < Q; av++) sum[av] = 0.0;
      for (int64_t k = k0 + lane; k < k1; k += 32) {
#pragma unroll
        for (int av = 0; av < Q; av++) sum[av] += load_s<double>(f[row[av] + k]);
      }
      // butterfly sums: every lane ends with all Q row sums; lane av keeps its own
#pragma unroll
      for (int av = 0; av < Q; av++) {
        double v = sum[av];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (av == lane) Sa = v;
      }
    } else {
      // FP32 storage values summed without rounding error as hi + lo pairs
      // (error-free TwoSum), so that only one FP64 addition per direction
      // remains (FP64 throughput is a small fraction of FP32 throughput here)
      float hi[Q], lo[Q];
#pragma unroll
      for (int av = 0; av < Q; av++) hi[av] = lo[av] = 0.f;
      for (int64_t k = k0 + lane; k < k1; k += 32) {
#pragma unroll
        for (int av = 0; av < Q; av++) two_sum_acc(hi[av], lo[av], load_s<float>(f[row[av] + k]));
      }
#pragma unroll
      for (int av = 0; av < Q; av++) {
        float h = hi[av], l = lo[av];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
          two_sum_acc(h, l, h2);
          l += l2;
        }
        if (av == lane) Sa = (double)h + (double)l;
      }
    }
    // weigh the column's Q sums, lane av taking direction av
    double part[7] = {0, 0, 0, 0, 0, 0, 0};
    const int av = lane;
    if (av < Q) {
      const int8_t *cv = dir_table<Q>(av);
      const bool crs = crosses_rt<Q>(ad, cv);
      int64_t r = c0;   // the column one step back along the slow axes of c_a
#pragma unroll
      for (int d = 0; d < D - 1; d++) {
        if (cv[d] < 0) r += ad.dp[d];
        if (cv[d] > 0) r += ad.dm[d];
      }
      const bool own = !ODD || av == 0 || crs;
      const int sl = own ? av : (av <= Lat<Q>::H ? av + Lat<Q>::H : av - Lat<Q>::H);
      const int64_t sc0 = own ? c0 : r;
      // the stored rows hold deviations from the reference of their locations
      Sa += (double)(k1 - k0) * ref_at<Q>(a.ref, sl, sc0);
      part[0] = Sa;
      if (av != 0) {
        double e[D], eb[D];
#pragma unroll
        for (int d = 0; d < D; d++) {
          double v = 0.0, vb = 0.0;
#pragma unroll
          for (int i = 0; i < D; i++) {
            v += cv[i] * a.gl[(c0 * D + i) * D + d];
            vb += cv[i] * a.gl[(r * D + i) * D + d];
          }
          e[d] = v;
          eb[d] = vb;
        }
        if (crs) {
#pragma unroll
          for (int d = 0; d < D; d++) eb[d] = e[d];
        } else {
#pragma unroll
          for (int ax = 0; ax < D - 1; ax++) {
            if (!a.has_rot[ax] || !a.periodic[ax] || cv[ax] == 0) continue;
            const bool below = cv[ax] > 0 && ad.ic[ax] == 0;
            const bool above = cv[ax] < 0 && ad.ic[ax] == a.g.n[ax] - 1;
            if (!below && !above) continue;
            double y[D];
            rot_vec<D>(a.rot[ax], above, eb, y);
#pragma unroll
            for (int d = 0; d < D; d++) eb[d] = y[d];
          }
        }
#pragma unroll
        for (int d = 0; d < D; d++) {
          part[1 + d] = e[d] * Sa;
          part[4 + d] = 0.5 * (e[d] + eb[d]) * Sa;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 7; k++) acc[k] += part[k];
  }
  block_sum<7>(acc, partial + (int64_t)blockIdx.x * 7);
}

// Any mesh, cell by cell: M is regrouped so that a cell needs only its own
// tangents. Substituting p = q - c_a in the second half of M,
//   M = 1/2 sum_p sum_a e*_a(p) [N_a(p) + N_a(p + c_a)]
// where the second population is left out when p + c_a lies behind a wall,
// N_a(p) is counted once more when p - c_a lies behind a wall (the reading
// e_a(q - c_a) := e_a(q) there), and e*_a(p) is e_a(p) rotated when the link
// p -> p + c_a crosses a seam with a rotation. Without rotations e*_a = e_a =
// c^i_a g_i(p), so the sums over directions collapse into
// B^i = sum_a c^i_a W_a and M_p = 1/2 g_i(p) B^i (P_p likewise): additions, and
// D x D products per cell. Under the A-A layout, N_a(p + c_a) sits at slot a of
// p + c_a (even parity) or at slot abar of p itself (odd parity).
template <int Q, typename S, bool ODD>
__global__ void __launch_bounds__(kMomThreads) k_totals_cells(const TotArgs a, double *partial) {
  constexpr int D = Lat<Q>::D;
  const S *f = static_cast<const S *>(a.f);
  const bool anyrot = a.has_rot[0] || a.has_rot[1] || a.has_rot[2];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const Addr<Q> ad(a.g, c);
    double N[Q];
    pull_abs<Q, ODD, S>(f, a.ncell, ad, a.ref, N);
    double gl[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
      for (int d = 0; d < D; d++) gl[i][d] = a.gl[(c * D + i) * D + d];
    double BP[D], BM[D];
#pragma unroll
    for (int i = 0; i < D; i++) BP[i] = BM[i] = 0.0;
    double mass = N[0];
#pragma unroll
    for (int av = 1; av < Q; av++) {
      mass += N[av];
      double W = N[av];
      if (ad.crosses(av, -1)) W += N[av];
      bool rotated = false;
      if (!ad.crosses(av, 1)) {
        const double Nn = ODD ? loc_abs<Q, S>(f, a.ncell, a.ref, lat_opp<Q>(av), c)
                              : loc_abs<Q, S>(f, a.ncell, a.ref, av, ad.nb(av, 1));
        if (anyrot) {
#pragma unroll
          for (int ax = 0; ax < D; ax++) {
            const int cax = Lat<Q>::c(av, ax);
            if (a.has_rot[ax] && a.periodic[ax] &&
                ((cax > 0 && ad.ic[ax] == a.g.n[ax] - 1) || (cax < 0 && ad.ic[ax] == 0)))
              rotated = true;
          }
        }
        if (!rotated) {
          W += Nn;
        } else {
          // e*_a: e_a(p) carried across the seam(s) of the link p -> p + c_a
          double e[D], y[D];
#pragma unroll
          for (int d = 0; d < D; d++) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < D; i++) v += Lat<Q>::c(av, i) * gl[i][d];
            e[d] = v;
          }
#pragma unroll
          for (int ax = 0; ax < D; ax++) {
            const int cax = Lat<Q>::c(av, ax);
            if (!a.has_rot[ax] || !a.periodic[ax]) continue;
            // seen from p + c_a, p is the image at index -1 (R^T) or n (R)
            const bool below = cax > 0 && ad.ic[ax] == a.g.n[ax] - 1;
            const bool above = cax < 0 && ad.ic[ax] == 0;
            if (!below && !above) continue;
            rot_vec<D>(a.rot[ax], above, e, y);
#pragma unroll
            for (int d = 0; d < D; d++) e[d] = y[d];
          }
#pragma unroll
          for (int d = 0; d < D; d++) acc[4 + d] += 0.5 * e[d] * Nn;
        }
      }
#pragma unroll
      for (int i = 0; i < D; i++) {
        const int ci = Lat<Q>::c(av, i);
        if (ci > 0) {
          BP[i] += N[av];
          BM[i] += W;
        }
        if (ci < 0) {
          BP[i] -= N[av];
          BM[i] -= W;
        }
      }
    }
    acc[0] += mass;
#pragma unroll
    for (int d = 0; d < D; d++) {
      double p = 0.0, m = 0.0;
#pragma unroll
      for (int i = 0; i < D; i++) {
        p += gl[i][d] * BP[i];
        m += gl[i][d] * BM[i];
      }
      acc[1 + d] += p;
      acc[4 + d] += 0.5 * m;
    }
  }
  block_sum<7>(acc, partial + (int64_t)blockIdx.x * 7);
}

template <int Q, typename S>
static cudaError_t totals_t(const vlb_sim *sim, double *d_partial, int64_t nblk_max, int64_t *nblk,
                            cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  const int dim = m->md.dim;
  TotArgs a;
  a.f = sim->d_f;
  a.g = make_grid(m);
  a.ncell = m->ncell;
  a.nfast = m->md.n[dim - 1];
  a.ncol = m->ncell / a.nfast;
  a.gl = m->d_gl;
  a.ref = make_ref(sim);
  for (int d = 0; d < 3; d++) {
    a.has_rot[d] = m->md.has_rot[d];
    a.periodic[d] = (d < dim && m->md.bc[d] == VLB_PERIODIC) ? 1 : 0;
    for (int k = 0; k < 9; k++) a.rot[d][k] = m->md.rot[d][k];
  }
  const bool odd = sim->t & 1;
  const bool columns = sim->plane && a.periodic[dim - 1] && !a.has_rot[dim - 1];
  if (columns) {
    const int64_t items = a.ncol * ((a.nfast + kTotChunk - 1) / kTotChunk);
    *nblk = std::min<int64_t>(nblk_max, (items + kMomThreads / 32 - 1) / (kMomThreads / 32));
    if (odd)
      k_totals_plane<Q, S, true><<<(unsigned)*nblk, kMomThreads, 0, s>>>(a, d_partial);
    else
      k_totals_plane<Q, S, false><<<(unsigned)*nblk, kMomThreads, 0, s>>>(a, d_partial);
  } else {
    *nblk = std::min<int64_t>(nblk_max, (a.ncell + kMomThreads - 1) / kMomThreads);
    if (odd)
      k_totals_cells<Q, S, true><<<(unsigned)*nblk, kMomThreads, 0, s>>>(a, d_partial);
    else
      k_totals_cells<Q, S, false><<<(unsigned)*nblk, kMomThreads, 0, s>>>(a, d_partial);
  }
  return cudaGetLastError();
}

cudaError_t launch_totals(const vlb_sim *sim, double *d_partial, int64_t nblk_max, double *d_totals,
                          cudaStream_t s) {
  int64_t nblk = 0;
  cudaError_t e = with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return sim->mesh->md.q == 9 ? totals_t<9, S>(sim, d_partial, nblk_max, &nblk, s)
                                : totals_t<19, S>(sim, d_partial, nblk_max, &nblk, s);
  });
  if (e != cudaSuccess) return e;
  return launch_finish_totals(d_partial, nblk, d_totals, s);
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

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
// Each thread writes exactly the locations it read, so no two threads touch
// the same word. Walls (index-space halfway bounce-back) fold into the same
// addressing: a population that would leave through a wall is written to the
// cell's own slot that the next step reads as the reflected arrival.
//
// The kernel is persistent: each block walks a contiguous run of tiles (128
// consecutive cells along the fastest axis), and each thread copies the Q
// populations of its cell in the NEXT tile into shared memory with
// asynchronous copies before it collides its cell in the current tile. The
// DRAM latency of the reads is thereby hidden behind a tile's worth of
// arithmetic without holding the loads in registers. A thread only ever
// reads the shared-memory slots it filled itself, so no block barrier is
// needed; and since the read and write sets of different cells are disjoint,
// reading tile k + 1 ahead of the writes of tile k is safe.
#include <mutex>
#include <tuple>
#include <vector>

#include "vlb_addr.cuh"
#include "vlb_collide.cuh"

namespace vlb {

struct StepArgs {
  void *f;
  const void *coef;
  int *err;
  Grid g;
  int64_t ncell;
  int32_t plane;    // one coefficient record per column of the fastest axis
  double tau, tol;
  double nref;      // populations are stored as N_a - w_a nref
  int32_t max_iter;
  int32_t moving;
  // tiles: index t = (A nB + B) ntf + tf over the two slow axes (A, B) and
  // the tiles tf of the fastest axis; 3D: (A, B) = (i0, i1); 2D: (0, i0)
  int64_t ntiles;
  int32_t ntf, nA, nB;
  int64_t per_block;  // tiles per block (contiguous runs)
};

constexpr int kStepThreads = 128;

// asynchronous global -> shared copies of one element (4 or 8 bytes)
template <int BYTES>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// position of a tile in the (A, B, tf) mixed radix
struct TileCursor {
  int32_t A, B, tf;
  __device__ __forceinline__ void set(int64_t t, const StepArgs &a) {
    tf = (int32_t)(t % a.ntf);
    const int64_t r = t / a.ntf;
    B = (int32_t)(r % a.nB);
    A = (int32_t)(r / a.nB);
  }
  __device__ __forceinline__ void next(const StepArgs &a) {
    if (++tf == a.ntf) {
      tf = 0;
      if (++B == a.nB) {
        B = 0;
        ++A;
      }
    }
  }
};

template <int Q, typename IT>
__device__ __forceinline__ Addr<Q, IT> tile_addr(const Grid &g, const TileCursor &c, IT ifast) {
  return Lat<Q>::D == 3 ? Addr<Q, IT>(g, (IT)c.A, (IT)c.B, ifast) : Addr<Q, IT>(g, (IT)c.B, ifast, (IT)0);
}

// index of the arrived population N_a(q, t) (the A-A read side): slot a of q
// (even parity, the rest population, or a link that comes back from a wall)
// or slot abar of q - c_a
template <int Q, bool ODD, typename IT>
__device__ __forceinline__ IT src_index(IT ps, const Addr<Q, IT> &ad, int a) {
  if (!ODD || a == 0 || ad.crosses(a, -1)) return (IT)a * ps + ad.cell;
  return (IT)lat_opp<Q>(a) * ps + ad.nb(a, -1);
}

template <typename R>
constexpr int step_min_blocks() {
  return sizeof(R) == 4 ? 4 : 2;
}

template <int Q, typename S, typename R, bool ODD, typename IT>
__global__ void __launch_bounds__(kStepThreads, step_min_blocks<R>()) k_step(const StepArgs a) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  using L = CoefLayout<Q>;
  constexpr int RS = L::template stride<R>();
  __shared__ S buf[2][Q][kStepThreads];
  const int64_t t0 = (int64_t)blockIdx.x * a.per_block;
  const int64_t t1 = t0 + a.per_block < a.ntiles ? t0 + a.per_block : a.ntiles;
  if (t0 >= t1) return;
  S *__restrict__ f = static_cast<S *>(a.f);
  const R *__restrict__ coef = static_cast<const R *>(a.coef);
  const IT ps = (IT)a.ncell;
  const IT nfast = (IT)(D == 3 ? a.g.n[2] : a.g.n[1]);
  const int tid = threadIdx.x;

  // issue the copies of this thread's cell in tile c into stage st
  auto prefetch = [&](const TileCursor &c, int st) {
    const IT ifast = (IT)c.tf * kStepThreads + (IT)tid;
    if (ifast < nfast) {
      const Addr<Q, IT> ad = tile_addr<Q, IT>(a.g, c, ifast);
#pragma unroll
      for (int av = 0; av < Q; av++) cp_async<sizeof(S)>(&buf[st][av][tid], f + src_index<Q, ODD, IT>(ps, ad, av));
    }
    cp_async_commit();
  };

  TileCursor cur, nxt;
  cur.set(t0, a);
  nxt = cur;
  prefetch(cur, 0);
  for (int64_t t = t0; t < t1; t++) {
    const int st = (int)((t - t0) & 1);
    nxt.next(a);
    if (t + 1 < t1)
      prefetch(nxt, st ^ 1);
    else
      cp_async_commit();
    cp_async_wait<1>();  // the copies of tile t are complete

    const IT ifast = (IT)cur.tf * kStepThreads + (IT)tid;
    if (ifast < nfast) {
      const Addr<Q, IT> ad = tile_addr<Q, IT>(a.g, cur, ifast);
      const IT cell = ad.cell;
      // ---- pull (read side of Eq. 22): deviations d_a = N_a - w_a n_ref
      R N[Q];
#pragma unroll
      for (int av = 0; av < Q; av++) N[av] = static_cast<R>(buf[st][av][tid]);

      // ---- coefficients: one record per column of the fastest axis (plane
      // mode), the same for every thread of the tile, or one per cell
      const IT rec = a.plane ? (IT)cur.A * (IT)a.nB + (IT)cur.B : cell;
      const R *__restrict__ rc = coef + (int64_t)rec * RS;

      // ---- collide (section 2.2)
      R Np[Q];
      CollideState<Q, R> cst;
      collide_cell<Q, R, true, true>(N, rc, R(a.nref), R(a.tau), R(a.tol), a.max_iter, Np, cst);
      if (!cst.conv) atomicOr(a.err, ERR_NOCONV);

      // ---- moving walls: a reflected population is corrected by
      //      -J rho [f^eq_a - f^eq_abar](rho = 1, U = U~ = U_wall)
      const bool moving = a.moving && ad.wall_cell();
      R uw[D];
#pragma unroll
      for (int i = 0; i < D; i++) uw[i] = moving ? rc[L::UW + i] : R(0);
      EqParts<Q, R> ew;
      if (moving) {
        R zero[D], gd[L::NS];
#pragma unroll
        for (int i = 0; i < D; i++) zero[i] = R(0);
#pragma unroll
        for (int i = 0; i < L::NS; i++) gd[i] = rc[L::GINV + i];
        eq_parts<Q, R>(gd, uw, zero, ew);
      }
      const R Jc = moving ? rc[L::J] : R(0);

      // ---- push (write side of Eq. 22)
#pragma unroll
      for (int av = 1; av < Q; av++) {
        const int ab = lat_opp<Q>(av);
        const bool crs = ad.crosses(av, 1);
        R v = Np[av];
        if (moving && crs) {
          const int p = av <= H ? av : av - H;
          const R O = eq_odd<Q, R>(ew, uw, p);
          const R corr = R(2) * Jc * cst.rho * lat_w<Q, R>(av) * O;
          v -= (av <= H) ? corr : -corr;
        }
        if (!ODD || crs)
          f[(IT)ab * ps + cell] = static_cast<S>(v);
        else
          f[(IT)av * ps + ad.nb(av, 1)] = static_cast<S>(v);
      }
      f[cell] = static_cast<S>(Np[0]);
    }
    cur = nxt;
  }
  cp_async_wait<0>();
}

// blocks the persistent kernel can keep resident on the current device
// (queried once per kernel and device)
static int resident_blocks(const void *kern) {
  static std::mutex mu;
  static std::vector<std::tuple<const void *, int, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (const auto &e : cache)
    if (std::get<0>(e) == kern && std::get<1>(e) == dev) return std::get<2>(e);
  int nb = 0, nsm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kStepThreads, 0);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int total = (nb > 0 ? nb : 1) * (nsm > 0 ? nsm : 1);
  cache.emplace_back(kern, dev, total);
  return total;
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
  a.ntf = (int32_t)((nfast + kStepThreads - 1) / kStepThreads);
  a.nA = (int32_t)(dim == 3 ? m->md.n[0] : 1);
  a.nB = (int32_t)(dim == 3 ? m->md.n[1] : m->md.n[0]);
  a.ntiles = (int64_t)a.ntf * a.nA * a.nB;
  // 32-bit indexing when every population offset fits
  const bool i32 = (int64_t)Q * m->ncell < ((int64_t)1 << 31);
  if (a.ntiles == 0) return cudaSuccess;
  auto go = [&](void (*kern)(StepArgs)) {
    const int64_t nblk_max = resident_blocks(reinterpret_cast<const void *>(kern));
    a.per_block = (a.ntiles + nblk_max - 1) / nblk_max;
    const int64_t nblk = (a.ntiles + a.per_block - 1) / a.per_block;
    kern<<<(unsigned)nblk, kStepThreads, 0, s>>>(a);
  };
  if (i32) {
    if (odd)
      go(k_step<Q, S, R, true, int32_t>);
    else
      go(k_step<Q, S, R, false, int32_t>);
  } else {
    if (odd)
      go(k_step<Q, S, R, true, int64_t>);
    else
      go(k_step<Q, S, R, false, int64_t>);
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

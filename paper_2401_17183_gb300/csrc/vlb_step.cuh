// vlb_step.cuh -- the fused stream-and-collide time step (Eq. 12 with the
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
// populations of its cell in tile k + 2 into shared memory with asynchronous
// copies while it collides its cell in tile k (three stages); on even steps of
// full tiles, where every direction reads the tile's own row segment, the
// block copies the Q segments in 16-byte pieces instead. The DRAM latency
// of the reads is thereby hidden behind the arithmetic of a tile without
// holding the loads in registers. In plane mode the tile's shared coefficient
// record travels in the same copy group, in 16-byte pieces; one block barrier
// per tile makes those pieces visible to every thread and guards the reuse of
// a stage. Since the read and write sets of different cells are disjoint,
// reading tile k + 2 ahead of the writes of tile k is safe.
//
// Populations may be stored in 16 bits (IEEE half or bfloat16) with FP32
// arithmetic: on even steps of full tiles the row segments are staged as
// they are; otherwise each value is staged as the aligned 32-bit word that
// contains it and the thread remembers which half it is.
#pragma once

#include <mutex>
#include <tuple>
#include <type_traits>
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
  double itau;      // 1 / tau
  // the same scalars rounded once for FP32 arithmetic, so that no cell
  // converts them
  float nref_f, itau_f, tol_f;
  int32_t max_iter;
  int32_t moving;
  // tiles: index t = (A nB + B) ntf + tf over the two slow axes (A, B) and
  // the tiles tf of the fastest axis; 3D: (A, B) = (i0, i1); 2D: (0, i0)
  int64_t ntiles;
  int32_t ntf, nA, nB;
  int64_t per_block;  // tiles per block (contiguous runs)
  int32_t full_tiles; // the fastest axis is a whole number of tiles
  // offsets of the population slots, k ncell and k ncell / 2 (32-bit words
  // of 16-bit storage), when every offset fits in 32 bits (else unused):
  // read by the kernel as constants, not formed per cell and direction
  int32_t soff[19], soffw[19];
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

// a step argument in the arithmetic type: the FP64 value or its FP32 copy
template <typename R>
__device__ __forceinline__ R arg_r(double v, float vf);
template <>
__device__ __forceinline__ double arg_r<double>(double v, float) {
  return v;
}
template <>
__device__ __forceinline__ float arg_r<float>(double, float vf) {
  return vf;
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

// does c_a move along a slow axis (and so, in plane mode, to another column)?
template <int Q>
__host__ __device__ constexpr bool slow_move(int a) {
  bool m = false;
  for (int d = 0; d < Lat<Q>::D - 1; d++) m = m || Lat<Q>::c(a, d) != 0;
  return m;
}

// resident blocks per SM the register budget is cut for: 3 for FP32
// storage (168 registers, no spills; 4 blocks at 128 registers ran 0.4%
// slower, 5 at 102 registers 18% slower), 4 for 16-bit storage (128
// registers; 3% faster than 3 blocks on even steps, 0.3% faster over both
// parities), 2 for FP64
template <typename R, typename S = R, bool ODD = false>
constexpr int step_min_blocks() {
  return sizeof(R) == 4 ? (sizeof(S) == 2 ? 4 : 3) : 2;
}

// pipeline depth: tiles whose copies are in flight while one is collided
constexpr int kStages = 3;

// Shared memory of one block: per stage, the populations of its 128 cells and,
// in plane mode, the coefficient record they all share. A 16-bit population
// is staged as the aligned 32-bit word that holds it (asynchronous copies move
// 4, 8 or 16 bytes), with one bit per direction saying which half it is.
// T is the tile width (threads per block).
template <int Q, typename S, typename R, int T = kStepThreads>
struct StepSmem {
  static constexpr int RS = CoefLayout<Q>::template stride<R, true>();
  static constexpr bool H16 = sizeof(S) == 2;
  using PopT = typename std::conditional<H16, uint32_t, S>::type;
  alignas(16) R rec[kStages][RS];
  PopT pop[kStages][Q][T];
  uint32_t half_hi[H16 ? kStages : 1][T];
};

// a 16-bit storage value from its bit pattern
template <typename S>
__device__ __forceinline__ S s16_from_bits(unsigned short b);
template <>
__device__ __forceinline__ __half s16_from_bits<__half>(unsigned short b) {
  return __ushort_as_half(b);
}
template <>
__device__ __forceinline__ __nv_bfloat16 s16_from_bits<__nv_bfloat16>(unsigned short b) {
  return __ushort_as_bfloat16(b);
}

// REFOFS: 16-bit populations stored relative to the rest state of the column
// that holds them (plane mode only); the collision works on them relative to
// its own column's rest state, so even steps add no offsets at all and odd
// steps add the record's column differences on links that change column.
// HPAR: 16-bit storage with an even cell count and an even fastest axis, so
// that which half of its 32-bit word a value sits in follows from the cell's
// own parity: a neighbour along a slow axis (or behind a wall: the own cell)
// has the same parity, one along the fastest axis (periodic wrap included:
// nfast - 1 is odd) the other one.
// The tiles [t0, t1) of one mesh, as one block of T threads (tiles of T
// cells; the arguments' tile counts must be those of width T).
// TAB: the slot offsets come from the argument table (the arguments are
// kernel parameters, so each offset is a constant operand) rather than from a
// product per cell and direction; only with 32-bit offsets.
// Cells away from every wall (on odd steps) index their neighbours with no
// wall test and no select: every move is a plain or a periodic one.
template <int Q, typename S, typename R, bool ODD, bool PLANE, bool REFOFS, bool HPAR, typename IT,
          int T = kStepThreads, bool TAB = true>
__device__ __forceinline__ void step_tiles(const StepArgs &a, const int64_t t0, const int64_t t1) {
  constexpr int D = Lat<Q>::D, H = Lat<Q>::H;
  static_assert(Q <= 19, "the slot-offset table holds 19 directions");
  constexpr bool USE_TAB = TAB && sizeof(IT) == 4;
  using L = CoefLayout<Q>;
  constexpr int RS = L::template stride<R, PLANE>();
  constexpr bool H16 = sizeof(S) == 2;
  static_assert(!REFOFS || (PLANE && H16), "storage offsets need plane mode and 16-bit storage");
  static_assert(!HPAR || H16, "half parity applies to 16-bit storage");
  // 16-byte pieces of the record that the kernel reads
  constexpr int RCHUNK = (REFOFS ? RS : L::SREST) * (int)sizeof(R) / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<Q, S, R, T> &sm = *reinterpret_cast<StepSmem<Q, S, R, T> *>(smem_raw);
  S *__restrict__ f = static_cast<S *>(a.f);
  const R *__restrict__ coef = static_cast<const R *>(a.coef);
  const IT ps = (IT)a.ncell;
  const IT nfast = (IT)(D == 3 ? a.g.n[2] : a.g.n[1]);
  const int tid = threadIdx.x;

  // pieces of 16 bytes in one direction's row segment of a tile
  constexpr int PER_ROW = T * (int)sizeof(S) / 16;

  // offset of slot k in elements (soff) and in 32-bit words of 16-bit
  // storage (soffw)
  auto soff = [&](int k) -> IT {
    if constexpr (USE_TAB)
      return (IT)a.soff[k];
    else
      return (IT)k * ps;
  };
  auto soffw = [&](int k) -> IT {
    if constexpr (USE_TAB)
      return (IT)a.soffw[k];
    else
      return (IT)k * (ps / 2);
  };
  // index of the arrived population N_a(q, t) (the A-A read side): slot a of
  // q (even parity, the rest population, or a link that comes back from a
  // wall) or slot abar of q - c_a; WALLS false: q is known to be away from
  // every wall. ws: the slot offsets to use (elements or words).
  auto src_idx = [&](const Addr<Q, IT> &ad, int av, auto walls_tag, auto ws) -> IT {
    constexpr bool WALLS = decltype(walls_tag)::value;
    if (!ODD || av == 0 || (WALLS && ad.crosses(av, -1))) return ws(av) + ad.cell;
    return ws(lat_opp<Q>(av)) + ad.nb(av, -1);
  };
  const std::true_type walls_yes;
  const std::false_type walls_no;

  // issue this thread's copies for tile c into stage st: the populations of
  // its cell and, in plane mode, one 16-byte piece of the shared record. On
  // even steps of full tiles every direction reads the tile's own row
  // segment, so the block copies the Q segments in 16-byte pieces instead
  // (thread tid takes pieces tid, tid + 128, ...).
  auto prefetch = [&](const TileCursor &c, int st) {
    const IT ifast = (IT)c.tf * T + (IT)tid;
    bool rows = false;
    if constexpr (!ODD) {
      if (a.full_tiles) {
        rows = true;
        const IT cell0 = tile_addr<Q, IT>(a.g, c, (IT)c.tf * T).cell;
#pragma unroll
        for (int k = tid; k < Q * PER_ROW; k += T) {
          const int av = k / PER_ROW, j = k - av * PER_ROW;
          cp_async<16>(reinterpret_cast<unsigned char *>(&sm.pop[st][av][0]) + 16 * j,
                       reinterpret_cast<const unsigned char *>(f + ((IT)av * ps + cell0)) + 16 * j);
        }
      }
    }
    if (!rows && ifast < nfast) {
      const Addr<Q, IT> ad = tile_addr<Q, IT>(a.g, c, ifast);
      if constexpr (H16 && HPAR) {
        // the same neighbour arithmetic on 32-bit words: the slow-axis moves
        // are even, the fastest-axis move is the cell's own word difference
        Addr<Q, IT> adw = ad;
        adw.cell = ad.cell >> 1;
#pragma unroll
        for (int d = 0; d < D - 1; d++) {
          adw.dp[d] = ad.dp[d] / 2;
          adw.dm[d] = ad.dm[d] / 2;
        }
        adw.dp[D - 1] = ((ad.cell + ad.dp[D - 1]) >> 1) - adw.cell;
        adw.dm[D - 1] = ((ad.cell + ad.dm[D - 1]) >> 1) - adw.cell;
        const uint32_t *fw = reinterpret_cast<const uint32_t *>(f);
        if (ODD && !ad.wall_cell()) {
#pragma unroll
          for (int av = 0; av < Q; av++) cp_async<4>(&sm.pop[st][av][tid], fw + src_idx(adw, av, walls_no, soffw));
        } else {
#pragma unroll
          for (int av = 0; av < Q; av++) cp_async<4>(&sm.pop[st][av][tid], fw + src_idx(adw, av, walls_yes, soffw));
        }
      } else if constexpr (H16) {
        uint32_t hi = 0;
#pragma unroll
        for (int av = 0; av < Q; av++) {
          const IT idx = src_idx(ad, av, walls_yes, soff);
          cp_async<4>(&sm.pop[st][av][tid], reinterpret_cast<const uint32_t *>(f) + (idx >> 1));
          hi |= (uint32_t)(idx & 1) << av;
        }
        sm.half_hi[st][tid] = hi;
      } else {
        if (ODD && !ad.wall_cell()) {
#pragma unroll
          for (int av = 0; av < Q; av++) cp_async<sizeof(S)>(&sm.pop[st][av][tid], f + src_idx(ad, av, walls_no, soff));
        } else {
#pragma unroll
          for (int av = 0; av < Q; av++) cp_async<sizeof(S)>(&sm.pop[st][av][tid], f + src_idx(ad, av, walls_yes, soff));
        }
      }
    }
    if constexpr (PLANE) {
      const int64_t rec = (int64_t)c.A * a.nB + c.B;
      // one piece per thread, or several where the block is narrower
      for (int k = tid; k < RCHUNK; k += T)
        cp_async<16>(reinterpret_cast<unsigned char *>(&sm.rec[st][0]) + 16 * k,
                     reinterpret_cast<const unsigned char *>(coef + rec * RS) + 16 * k);
    }
  };

  // prologue: tiles t0 .. t0 + kStages - 2, one copy group each
  TileCursor cur, nxt;
  cur.set(t0, a);
  nxt = cur;
#pragma unroll
  for (int k = 0; k < kStages - 1; k++) {
    if (t0 + k < t1) prefetch(nxt, k);
    cp_async_commit();
    nxt.next(a);
  }
  int st = 0;
  for (int64_t t = t0; t < t1; t++) {
    // the copies of tile t (this thread's) are complete; after the barrier
    // every thread's are, and every thread is done with tile t - 1, whose
    // stage the next prefetch reuses
    cp_async_wait<kStages - 2>();
    __syncthreads();
    {
      int sn = st + kStages - 1;
      if (sn >= kStages) sn -= kStages;
      if (t + kStages - 1 < t1) prefetch(nxt, sn);
      cp_async_commit();
      nxt.next(a);
    }

    const IT ifast = (IT)cur.tf * T + (IT)tid;
    if (ifast < nfast) {
      const Addr<Q, IT> ad = tile_addr<Q, IT>(a.g, cur, ifast);
      const IT cell = ad.cell;
      // ---- pull (read side of Eq. 22): deviations d_a = N_a - w_a n_ref
      // ---- coefficients: in plane mode one record per column of the fastest
      // axis, shared by the tile and staged in shared memory; else one per cell
      const R *__restrict__ rc = PLANE ? &sm.rec[st][0] : coef + (int64_t)cell * RS;

      R N[Q];
      if constexpr (H16) {
        if (!ODD && a.full_tiles) {
          // the tile's row segments, 16 bits per cell
#pragma unroll
          for (int av = 0; av < Q; av++)
            N[av] = load_s<R>(s16_from_bits<S>(reinterpret_cast<const unsigned short *>(&sm.pop[st][av][0])[tid]));
        } else {
          const uint32_t hi = HPAR ? 0u : sm.half_hi[st][tid];
          // HPAR: the shift of the own cell's half and of the other one
          const unsigned sh0 = ((unsigned)cell & 1u) << 4, sh1 = 16u - sh0;
          auto unpack = [&](auto inner_tag) {
            [[maybe_unused]] constexpr bool INNER = decltype(inner_tag)::value;
#pragma unroll
            for (int av = 0; av < Q; av++) {
              const uint32_t w = sm.pop[st][av][tid];
              unsigned short b;
              if constexpr (HPAR) {
                // away from walls every move along the fastest axis reads the
                // other half; a link through a wall reads the own cell
                const bool shifted = ODD && Lat<Q>::c(av, D - 1) != 0 && (INNER || !ad.crosses(av, -1));
                b = (unsigned short)(w >> (shifted ? sh1 : sh0));
              } else {
                b = (unsigned short)(((hi >> av) & 1) ? (w >> 16) : (w & 0xffffu));
              }
              N[av] = load_s<R>(s16_from_bits<S>(b));
            }
          };
          // a tile away from every wall (uniform over the tile): the halves
          // follow from the cell parity alone
          bool inner = ODD && HPAR && !a.g.wall[D - 1];
#pragma unroll
          for (int d = 0; d < D - 1; d++) inner = inner && !ad.lo[d] && !ad.hi[d];
          if (inner)
            unpack(std::true_type());
          else
            unpack(std::false_type());
        }
        if constexpr (REFOFS && ODD) {
          // relative to the own column's rest state: a population read from a
          // neighbouring column carries that column's storage reference. The
          // record's differences are zero where a slow-axis wall sends the link
          // back to the own slot; a fastest-axis wall does so only at the ends
          // of a row, which the masks take care of.
          const R mlo = ad.lo[D - 1] ? R(0) : R(1), mhi = ad.hi[D - 1] ? R(0) : R(1);
#pragma unroll
          for (int av = 1; av < Q; av++)
            if (slow_move<Q>(av)) {
              const int cz = Lat<Q>::c(av, D - 1);
              const R dv = rc[L::DIN + av];
              N[av] = cz == 0 ? N[av] + dv : fmar(dv, cz > 0 ? mlo : mhi, N[av]);
            }
        }
      } else {
#pragma unroll
        for (int av = 0; av < Q; av++) N[av] = static_cast<R>(sm.pop[st][av][tid]);
      }

      // ---- collide (section 2.2)
      R Np[Q];
      CollideState<Q, R> cst;
      // (with one record per cell the rest state is formed, not read)
      collide_cell<Q, R, true, REFOFS, PLANE>(N, rc, arg_r<R>(a.nref, a.nref_f), arg_r<R>(a.itau, a.itau_f),
                                     arg_r<R>(a.tol, a.tol_f), a.max_iter, Np, cst);
      if (!cst.conv) atomicOr(a.err, ERR_NOCONV);

      // ---- moving walls (wall cells only, one branch per cell): a reflected
      //      population is corrected by -J rho [f^eq_a - f^eq_abar](rho = 1,
      //      U = U~ = U_wall)
      if (a.moving && ad.wall_cell()) {
        R uw[D], zero[D], gd[L::NS];
#pragma unroll
        for (int i = 0; i < D; i++) {
          uw[i] = rc[L::UW + i];
          zero[i] = R(0);
        }
#pragma unroll
        for (int i = 0; i < L::NS; i++) gd[i] = R(2) * rc[L::GH + i];
        EqParts<Q, R> ew;
        eq_parts<Q, R>(gd, uw, zero, ew);
        const R Jr2 = R(2) * rc[L::J] * cst.rho;
#pragma unroll
        for (int av = 1; av < Q; av++) {
          const int p = av <= H ? av : av - H;
          const R corr = Jr2 * lat_w<Q, R>(av) * eq_odd<Q, R>(ew, uw, p);
          const R nv = Np[av] - ((av <= H) ? corr : -corr);
          Np[av] = ad.crosses(av, 1) ? nv : Np[av];
        }
      }

      // ---- push (write side of Eq. 22): own slot abar (even steps, and a
      //      link through a wall), else slot a of q + c_a; WALLS false: the
      //      cell is away from every wall
      auto push = [&](auto walls_tag) {
        constexpr bool WALLS = decltype(walls_tag)::value;
#pragma unroll
        for (int av = 1; av < Q; av++) {
          const int ab = lat_opp<Q>(av);
          const bool crs = WALLS && ad.crosses(av, 1);
          R v = Np[av];
          if constexpr (REFOFS && ODD) {
            if (slow_move<Q>(av)) {
              const int cz = Lat<Q>::c(av, D - 1);
              const R dv = rc[L::DOUT + av];
              if (WALLS)
                v = cz == 0 ? v + dv
                            : fmar(dv, cz > 0 ? (ad.hi[D - 1] ? R(0) : R(1)) : (ad.lo[D - 1] ? R(0) : R(1)), v);
              else
                v = v + dv;
            }
          }
          // one store through a selected index
          const IT idx = (!ODD || crs) ? soff(ab) + cell : soff(av) + ad.nb(av, 1);
          f[idx] = store_s<S>(v);
        }
      };
      if (ODD && !ad.wall_cell())
        push(walls_no);
      else
        push(walls_yes);
      f[cell] = store_s<S>(Np[0]);
    }
    cur.next(a);
    if (++st == kStages) st = 0;
  }
  cp_async_wait<0>();
}

// One mesh: block b walks the tiles [b per_block, (b + 1) per_block).
template <int Q, typename S, typename R, bool ODD, bool PLANE, bool REFOFS, bool HPAR, typename IT>
__global__ void __launch_bounds__(kStepThreads, step_min_blocks<R, S, ODD>())
    k_step(const __grid_constant__ StepArgs a) {
  const int64_t t0 = (int64_t)blockIdx.x * a.per_block;
  const int64_t t1 = t0 + a.per_block < a.ntiles ? t0 + a.per_block : a.ntiles;
  if (t0 >= t1) return;
  step_tiles<Q, S, R, ODD, PLANE, REFOFS, HPAR, IT>(a, t0, t1);
}

// Many meshes in one launch: block b takes the run of tiles items[b] of mesh
// items[b].sim, whose arguments are args[items[b].sim].
struct BatchItem {
  int32_t sim;
  int32_t pad;
  int64_t t0, t1;
};

// T threads per block (the tile width) and at least MINB resident blocks per
// SM (which caps the registers per thread): the batch's block shape.
template <int Q, typename S, typename R, bool ODD, bool PLANE, typename IT, int T, int MINB>
__global__ void __launch_bounds__(T, MINB)
    k_step_batch(const StepArgs *__restrict__ args, const BatchItem *__restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  // the arguments sit in global memory here: slot offsets are formed, not read
  step_tiles<Q, S, R, ODD, PLANE, false, false, IT, T, false>(args[it.sim], it.t0, it.t1);
}

// Arguments of one simulation's step kernel for tiles of T cells (per_block
// left for the caller).
template <int Q>
inline StepArgs make_step_args(const vlb_sim *sim, int T = kStepThreads) {
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
  a.itau = 1.0 / sim->p.tau;
  a.nref_f = (float)a.nref;
  a.itau_f = (float)a.itau;
  a.tol_f = (float)a.tol;
  a.max_iter = sim->p.max_iter;
  a.moving = 0;
  for (int ax = 0; ax < 3; ax++)
    for (int sd = 0; sd < 2; sd++)
      for (int d = 0; d < 3; d++)
        if (sim->p.wall_u[ax][sd][d] != 0.0 || sim->p.wall_omega[ax][sd][d] != 0.0) a.moving = 1;
  const int dim = m->md.dim;
  const int64_t nfast = dim == 3 ? m->md.n[2] : m->md.n[1];
  a.ntf = (int32_t)((nfast + T - 1) / T);
  a.nA = (int32_t)(dim == 3 ? m->md.n[0] : 1);
  a.nB = (int32_t)(dim == 3 ? m->md.n[1] : m->md.n[0]);
  a.ntiles = (int64_t)a.ntf * a.nA * a.nB;
  a.per_block = 0;
  a.full_tiles = nfast % T == 0 ? 1 : 0;
  const bool i32 = (int64_t)Q * m->ncell < ((int64_t)1 << 31);
  for (int k = 0; k < 19; k++) {
    a.soff[k] = (i32 && k < Q) ? (int32_t)(k * m->ncell) : 0;
    a.soffw[k] = (i32 && k < Q) ? (int32_t)(k * (m->ncell / 2)) : 0;
  }
  return a;
}

// blocks the persistent kernel can keep resident on the current device
// (queried once per kernel and device)
static int resident_blocks(const void *kern, size_t smem, int threads = kStepThreads) {
  static std::mutex mu;
  static std::vector<std::tuple<const void *, int, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (const auto &e : cache)
    if (std::get<0>(e) == kern && std::get<1>(e) == dev) return std::get<2>(e);
  int nb = 0, nsm = 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int total = (nb > 0 ? nb : 1) * (nsm > 0 ? nsm : 1);
  cache.emplace_back(kern, dev, total);
  return total;
}

template <int Q, typename S, typename R>
cudaError_t launch_step_t(const vlb_sim *sim, int odd, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  StepArgs a = make_step_args<Q>(sim);
  // 32-bit indexing when every population offset fits
  const bool i32 = (int64_t)Q * m->ncell < ((int64_t)1 << 31);
  if (a.ntiles == 0) return cudaSuccess;
  const size_t smem = sizeof(StepSmem<Q, S, R>);
  auto go = [&](void (*kern)(StepArgs)) {
    const int64_t nblk_max = resident_blocks(reinterpret_cast<const void *>(kern), smem);
    a.per_block = (a.ntiles + nblk_max - 1) / nblk_max;
    const int64_t nblk = (a.ntiles + a.per_block - 1) / a.per_block;
    kern<<<(unsigned)nblk, kStepThreads, smem, s>>>(a);
  };
  auto pick = [&](auto plane_tag, auto ref_tag, auto par_tag) {
    constexpr bool P = decltype(plane_tag)::value, RO = decltype(ref_tag)::value;
    constexpr bool HP = decltype(par_tag)::value;
    if (i32) {
      if (odd)
        go(k_step<Q, S, R, true, P, RO, HP, int32_t>);
      else
        go(k_step<Q, S, R, false, P, RO, HP, int32_t>);
    } else {
      if (odd)
        go(k_step<Q, S, R, true, P, RO, HP, int64_t>);
      else
        go(k_step<Q, S, R, false, P, RO, HP, int64_t>);
    }
  };
  const std::true_type yes;
  const std::false_type no;
  if constexpr (sizeof(S) == 2) {
    // the half of a 16-bit value follows from the cell parity when both the
    // cell count and the fastest axis are even
    const bool par = m->ncell % 2 == 0 && m->md.n[m->md.dim - 1] % 2 == 0;
    auto pick_par = [&](auto plane_tag, auto ref_tag) {
      if (par)
        pick(plane_tag, ref_tag, yes);
      else
        pick(plane_tag, ref_tag, no);
    };
    if (a.plane && sim->ref_rest)
      pick_par(yes, yes);
    else if (a.plane)
      pick_par(yes, no);
    else
      pick_par(no, no);
  } else {
    if (a.plane)
      pick(yes, no, no);
    else
      pick(no, no, no);
  }
  return cudaGetLastError();
}

}  // namespace vlb

// vlb_addr.cuh -- index arithmetic of the structured lattice: coordinates of
// a cell, its neighbours q +- c_a with periodic wrap, wall crossings, and the
// A-A read of the arrived populations N_a(q, t) for either layout parity.
#pragma once

#include "vlb_internal.cuh"

namespace vlb {

struct Grid {
  int64_t n[3];
  int64_t s[3];
  int32_t wall[3];
};

template <int Q, typename IT = int64_t>
struct Addr {
  static constexpr int D = Lat<Q>::D;
  IT cell;
  IT ic[3];
  IT dp[3], dm[3];
  bool lo[3], hi[3];

  // from a linear cell index (divisions; used outside the hot kernel)
  __device__ __forceinline__ Addr(const Grid &g, int64_t c) {
    int64_t r = c;
    ic[2] = (IT)(r % g.n[2]);
    r /= g.n[2];
    ic[1] = (IT)(r % g.n[1]);
    ic[0] = (IT)(r / g.n[1]);
    cell = (IT)c;
    init(g);
  }
  // from index coordinates
  __device__ __forceinline__ Addr(const Grid &g, IT i0, IT i1, IT i2) {
    ic[0] = i0;
    ic[1] = i1;
    ic[2] = i2;
    cell = (i0 * (IT)g.n[1] + i1) * (IT)g.n[2] + i2;
    init(g);
  }
  __device__ __forceinline__ void init(const Grid &g) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const IT n = (IT)g.n[d], st = (IT)g.s[d];
      dp[d] = (ic[d] == n - 1) ? -(n - 1) * st : st;
      dm[d] = (ic[d] == 0) ? (n - 1) * st : -st;
      lo[d] = g.wall[d] && ic[d] == 0;
      hi[d] = g.wall[d] && ic[d] == n - 1;
    }
  }
  __device__ __forceinline__ bool wall_cell() const {
    bool w = false;
#pragma unroll
    for (int d = 0; d < D; d++) w = w || lo[d] || hi[d];
    return w;
  }
  // does q + sg c_a leave the domain through a wall? (a, sg compile-time
  // constants after unrolling)
  __device__ __forceinline__ bool crosses(int a, int sg) const {
    bool x = false;
#pragma unroll
    for (int d = 0; d < D; d++) {
      const int cd = sg * Lat<Q>::c(a, d);
      if (cd > 0) x = x || hi[d];
      if (cd < 0) x = x || lo[d];
    }
    return x;
  }
  // linear index of q + sg c_a (periodic wrap on every axis)
  __device__ __forceinline__ IT nb(int a, int sg) const {
    IT r = cell;
#pragma unroll
    for (int d = 0; d < D; d++) {
      const int cd = sg * Lat<Q>::c(a, d);
      if (cd > 0) r += dp[d];
      if (cd < 0) r += dm[d];
    }
    return r;
  }
};

// Storage location (slot, cell) of the arrived population N_a(q, t). Even
// parity: slot a of q. Odd parity (the layout an even step leaves behind):
// slot abar of q - c_a, or slot a of q when q - c_a lies beyond a wall
// (halfway bounce-back).
template <int Q, bool ODD, typename IT>
__device__ __forceinline__ void arrived_loc(const Addr<Q, IT> &ad, int a, int &slot, IT &cell) {
  if (!ODD || a == 0 || ad.crosses(a, -1)) {
    slot = a;
    cell = ad.cell;
  } else {
    slot = lat_opp<Q>(a);
    cell = ad.nb(a, -1);
  }
}

// Arrived populations N_a(q, t) themselves, in FP64: the stored deviation
// plus the storage reference of its location.
template <int Q, bool ODD, typename S, typename IT>
__device__ __forceinline__ void pull_abs(const S *__restrict__ f, IT ps, const Addr<Q, IT> &ad,
                                         const RefCtx &ref, double (&N)[Q]) {
#pragma unroll
  for (int a = 0; a < Q; a++) {
    int slot;
    IT cell;
    arrived_loc<Q, ODD, IT>(ad, a, slot, cell);
    N[a] = load_s<double>(f[(IT)slot * ps + cell]) + ref_at<Q>(ref, slot, (int64_t)cell);
  }
}

inline Grid make_grid(const vlb_mesh *m) {
  Grid g;
  for (int d = 0; d < 3; d++) {
    g.n[d] = m->md.n[d];
    g.wall[d] = (d < m->md.dim && m->md.bc[d] == VLB_WALL) ? 1 : 0;
  }
  g.s[2] = 1;
  g.s[1] = g.n[2];
  g.s[0] = g.n[1] * g.n[2];
  return g;
}

}  // namespace vlb

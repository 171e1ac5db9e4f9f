// vlb_geometry.cu -- FP64 geometry precompute of section 2.1 (done once per
// mesh), mesh diagnostics, the coefficient records the step kernel streams,
// and the equilibrium initialisation of the populations.
#include <type_traits>

#include "vlb_addr.cuh"
#include "vlb_collide.cuh"
#include "vlb_q39.cuh"

namespace vlb {

// ------------------------------------------------------------------ positions
// y <- T_a^k (y), T_a(x) = R_a x + shift_a (inverse for k < 0)
__device__ __noinline__ void apply_period(const MeshDev &m, int ax, int64_t k, double y[3]) {
  const int D = m.dim;
  const double *R = m.rot[ax];
  const double *sh = m.shift[ax];
  for (int64_t t = 0; t < (k > 0 ? k : -k); t++) {
    double z[3] = {y[0], y[1], y[2]};
    if (k > 0) {
      if (m.has_rot[ax])
        for (int i = 0; i < D; i++) {
          double acc = 0.0;
          for (int j = 0; j < D; j++) acc += R[3 * i + j] * z[j];
          y[i] = acc;
        }
      for (int i = 0; i < D; i++) y[i] += sh[i];
    } else {
      for (int i = 0; i < D; i++) z[i] -= sh[i];
      if (m.has_rot[ax]) {
        for (int i = 0; i < D; i++) {
          double acc = 0.0;
          for (int j = 0; j < D; j++) acc += R[3 * j + i] * z[j];
          y[i] = acc;
        }
      } else {
        for (int i = 0; i < D; i++) y[i] = z[i];
      }
    }
  }
}

// position of p whose wall-axis coordinates are in range: wrap the periodic
// axes and apply the image transforms, axis 0 outermost
__device__ __noinline__ void position_periodic(const MeshDev &m, const int64_t p[3], double out[3]) {
  int64_t w[3], k[3];
  for (int a = 0; a < 3; a++) {
    w[a] = p[a];
    k[a] = 0;
    if (a < m.dim && m.bc[a] == VLB_PERIODIC) {
      int64_t q = p[a] / m.n[a];
      if (p[a] < 0 && q * m.n[a] != p[a]) q -= 1;  // floor division
      k[a] = q;
      w[a] = p[a] - q * m.n[a];
    }
  }
  const int64_t idx = (w[0] * m.n[1] + w[1]) * m.n[2] + w[2];
  for (int d = 0; d < 3; d++) out[d] = d < m.dim ? m.x[idx * m.dim + d] : 0.0;
  for (int a = m.dim - 1; a >= 0; a--)
    if (k[a] != 0) apply_period(m, a, k[a], out);
}

// position of any index p: behind a wall, linear extrapolation along that axis
// from the two nearest interior nodes, x(-k) = (1 + k) x(0) - k x(1)
__device__ __noinline__ void position(const MeshDev &m, const int64_t p[3], double out[3]) {
  int wa[3], nw = 0;
  int64_t b0[3], b1[3];
  double c0[3], c1[3];
  for (int a = 0; a < m.dim; a++) {
    if (m.bc[a] != VLB_WALL || (p[a] >= 0 && p[a] < m.n[a])) continue;
    const int64_t k = p[a] < 0 ? -p[a] : p[a] - (m.n[a] - 1);
    wa[nw] = a;
    b0[nw] = p[a] < 0 ? 0 : m.n[a] - 1;
    b1[nw] = p[a] < 0 ? 1 : m.n[a] - 2;
    c0[nw] = 1.0 + (double)k;
    c1[nw] = -(double)k;
    nw++;
  }
  out[0] = out[1] = out[2] = 0.0;
  for (int combo = 0; combo < (1 << nw); combo++) {
    int64_t pp[3] = {p[0], p[1], p[2]};
    double wgt = 1.0;
    for (int t = 0; t < nw; t++) {
      const bool second = (combo >> t) & 1;
      pp[wa[t]] = second ? b1[t] : b0[t];
      wgt *= second ? c1[t] : c0[t];
    }
    double y[3];
    position_periodic(m, pp, y);
    for (int d = 0; d < 3; d++) out[d] += wgt * y[d];
  }
}

__device__ __forceinline__ double nrm(const double v[3]) {
  return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

// tangent basis g_i(p) (Eqs. 1, 3); false on a folded arm (D_i = D_-i)
__device__ __noinline__ bool tangents(const MeshDev &m, const int64_t p[3], double gl[3][3]) {
  const double dx = m.dx > 0.0 ? m.dx : 1.0;
  double x0[3];
  position(m, p, x0);
  bool ok = true;
  for (int i = 0; i < 3; i++)
    for (int d = 0; d < 3; d++) gl[i][d] = 0.0;
  for (int i = 0; i < m.dim; i++) {
    int64_t pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
    pp[i] += 1;
    pm[i] -= 1;
    double xp[3], xm[3], Dp[3], Dm[3], df[3];
    position(m, pp, xp);
    position(m, pm, xm);
    for (int d = 0; d < 3; d++) {
      Dp[d] = xp[d] - x0[d];
      Dm[d] = xm[d] - x0[d];
      df[d] = Dp[d] - Dm[d];
    }
    const double nd = nrm(df);
    if (!(nd > 0.0)) {
      ok = false;
      continue;
    }
    const double beta = (nrm(Dp) + nrm(Dm)) / nd;
    for (int d = 0; d < 3; d++) gl[i][d] = beta * df[d] / (2.0 * dx);
  }
  return ok;
}

// J (Eq. 5) and co-tangents g^i (Eq. 7); in 2D the third tangent is z
__device__ __noinline__ bool dual(int dim, const double gl[3][3], double &J, double gu[3][3]) {
  for (int i = 0; i < 3; i++)
    for (int d = 0; d < 3; d++) gu[i][d] = 0.0;
  if (dim == 2) {
    J = gl[0][0] * gl[1][1] - gl[0][1] * gl[1][0];
    if (!(J > 0.0)) return false;
    gu[0][0] = gl[1][1] / J;
    gu[0][1] = -gl[1][0] / J;
    gu[1][0] = -gl[0][1] / J;
    gu[1][1] = gl[0][0] / J;
    return true;
  }
  double c12[3], c23[3], c31[3];
  auto cross = [](const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
  };
  cross(gl[0], gl[1], c12);
  cross(gl[1], gl[2], c23);
  cross(gl[2], gl[0], c31);
  J = c12[0] * gl[2][0] + c12[1] * gl[2][1] + c12[2] * gl[2][2];
  if (!(J > 0.0)) return false;
  for (int d = 0; d < 3; d++) {
    gu[0][d] = c23[d] / J;
    gu[1][d] = c31[d] / J;
    gu[2][d] = c12[d] / J;
  }
  return true;
}

// ------------------------------------------------------------------ precompute
template <int Q>
__global__ void k_geometry(const MeshDev m, Grid g, int64_t ncell, double *J_out, double *gl_out,
                           double *gu_out, double *ginv_out, double *K_out, int *err) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  const Addr<Q> ad(g, cell);
  const int64_t q[3] = {ad.ic[0], ad.ic[1], ad.ic[2]};
  double gl[3][3], gu[3][3], J = 0.0;
  bool ok = tangents(m, q, gl);
  ok = ok && dual(D, gl, J, gu);
  if (!ok) {
    atomicOr(err, ERR_GEOM);
    J = nan("");
  }
  J_out[cell] = J;
  for (int i = 0; i < D; i++)
    for (int d = 0; d < D; d++) {
      gl_out[(cell * D + i) * D + d] = gl[i][d];
      gu_out[(cell * D + i) * D + d] = gu[i][d];
    }
  for (int i = 0; i < D; i++)
    for (int j = i; j < D; j++) {
      double s = 0.0;
      for (int d = 0; d < 3; d++) s += gu[i][d] * gu[j][d];  // g^ij = g^i . g^j (Eq. 8)
      ginv_out[cell * NS + sym<D>(i, j)] = s;
    }
  for (int i = 0; i < D; i++) K_out[(cell * Q + 0) * D + i] = 0.0;
  // K^i_a = sum_j c^j_a [g_j(q + c_a) - g_j(q)] . g^i(q) = sum_j c^j_a Theta^i_j(q + c_a, q) (Eq. 11)
#pragma unroll 1
  for (int a = 1; a < Q; a++) {
    double Kv[3] = {0.0, 0.0, 0.0};
    // links that cross a wall: zero, or from the ghost-node tangents
    if (!ad.crosses(a, 1) || m.wall_links == VLB_WALL_LINKS_GHOST) {
      int64_t p[3] = {q[0], q[1], q[2]};
      for (int d = 0; d < D; d++) p[d] += Lat<Q>::c(a, d);
      double gp[3][3];
      if (!tangents(m, p, gp)) atomicOr(err, ERR_GEOM);
      double de[3] = {0.0, 0.0, 0.0};
      for (int j = 0; j < D; j++) {
        const int cj = Lat<Q>::c(a, j);
        if (cj == 0) continue;
        for (int d = 0; d < 3; d++) de[d] += cj * (gp[j][d] - gl[j][d]);
      }
      for (int i = 0; i < D; i++) Kv[i] = de[0] * gu[i][0] + de[1] * gu[i][1] + de[2] * gu[i][2];
    }
    for (int i = 0; i < D; i++) K_out[(cell * Q + a) * D + i] = Kv[i];
  }
}

cudaError_t launch_geometry(const vlb_mesh *m, int *d_err, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  const Grid g = make_grid(m);
  if (m->md.q == 9)
    k_geometry<9><<<(unsigned)blocks, threads, 0, s>>>(m->md, g, m->ncell, m->d_J, m->d_gl,
                                                       m->d_gu, m->d_ginv, m->d_K, d_err);
  else if (m->md.q == 39)
    k_geometry<39><<<(unsigned)blocks, threads, 0, s>>>(m->md, g, m->ncell, m->d_J, m->d_gl,
                                                        m->d_gu, m->d_ginv, m->d_K, d_err);
  else
    k_geometry<19><<<(unsigned)blocks, threads, 0, s>>>(m->md, g, m->ncell, m->d_J, m->d_gl,
                                                        m->d_gu, m->d_ginv, m->d_K, d_err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ diagnostics
// per block: [min J, -max J, min f^eq_rest/w, min g^ii, -max g^ii], reduced on the host
template <int Q>
__global__ void k_mesh_stats(const double *J, const double *ginv, int64_t ncell,
                             double *partial) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2, H = Lat<Q>::H;
  __shared__ double sh[5][kStatThreads];
  double v[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    v[0] = fmin(v[0], J[c]);
    v[1] = fmin(v[1], -J[c]);
    double gi[NS], gd[NS], U[D], Ut[D];
    for (int i = 0; i < NS; i++) gd[i] = gi[i] = ginv[c * NS + i];
    for (int i = 0; i < D; i++) gd[sym<D>(i, i)] -= 1.0;
    for (int i = 0; i < D; i++) U[i] = Ut[i] = 0.0;
    EqParts<Q, double> e;
    eq_parts<Q, double>(gd, U, Ut, e);
    double m = eq_even<Q, double>(e, 0);
#pragma unroll
    for (int p = 1; p <= H; p++) m = fmin(m, eq_even<Q, double>(e, p));
    v[2] = fmin(v[2], m);
    for (int i = 0; i < D; i++) {
      v[3] = fmin(v[3], gi[sym<D>(i, i)]);
      v[4] = fmin(v[4], -gi[sym<D>(i, i)]);
    }
  }
  for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; k++) partial[blockIdx.x * 5 + k] = sh[k][0];
}

cudaError_t launch_mesh_stats(const vlb_mesh *m, double *d_partial, int64_t nblk, cudaStream_t s) {
  if (m->md.q == 9)
    k_mesh_stats<9><<<(unsigned)nblk, kStatThreads, 0, s>>>(m->d_J, m->d_ginv, m->ncell, d_partial);
  else
    k_mesh_stats<19><<<(unsigned)nblk, kStatThreads, 0, s>>>(m->d_J, m->d_ginv, m->ncell, d_partial);
  return cudaGetLastError();
}

// plane check: does every cell's geometry equal that of the first cell of its
// column along the fastest axis (to 1e-12 relative)?
__device__ __forceinline__ bool close12(double a, double b) {
  return fabs(a - b) <= 1e-12 * (1.0 + fabs(b));
}

template <int Q>
__global__ void k_plane_check(const double *J, const double *ginv, const double *gu,
                              const double *K, int64_t ncell, int64_t nfast, int *flag) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int64_t c0 = (c / nfast) * nfast;
  if (c0 == c) return;
  bool same = close12(J[c], J[c0]);
  for (int i = 0; i < NS; i++) same = same && close12(ginv[c * NS + i], ginv[c0 * NS + i]);
  for (int i = 0; i < D * D; i++) same = same && close12(gu[c * D * D + i], gu[c0 * D * D + i]);
  for (int i = 0; i < Q * D; i++) same = same && close12(K[c * Q * D + i], K[c0 * Q * D + i]);
  if (!same) atomicOr(flag, 1);
}

cudaError_t launch_plane_check(const vlb_mesh *m, int *d_flag, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  const int64_t nfast = m->md.n[m->md.dim - 1];
  if (m->md.q == 9)
    k_plane_check<9><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_ginv, m->d_gu, m->d_K,
                                                          m->ncell, nfast, d_flag);
  else
    k_plane_check<19><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_ginv, m->d_gu, m->d_K,
                                                           m->ncell, nfast, d_flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ coefficient records
struct PackArgs {
  MeshDev md;
  Grid g;
  const double *J, *gu, *ginv, *K;
  int64_t nrec, stride, nfast;
  int32_t plane;
  double tau;
  double body[3];
  double wall_u[3][2][3];
  double wall_omega[3][2][3];
  int32_t ref_rest;  // fill the storage-reference offsets (16-bit storage, plane mode)
  double nref;
};

template <int Q, typename R>
__global__ void k_pack_coef(const PackArgs a, R *coef) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2, H = Lat<Q>::H;
  using L = CoefLayout<Q>;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.nrec) return;
  const int64_t c = a.plane ? r * a.nfast : r;
  double K[Q][D], G[D], rec[L::NC];
  for (int av = 0; av < Q; av++)
    for (int i = 0; i < D; i++) K[av][i] = a.K[(c * Q + av) * D + i];
  for (int i = 0; i < D; i++) {
    double s = 0.0;
    for (int d = 0; d < D; d++) s += a.body[d] * a.gu[(c * D + i) * D + d];  // G^i = G . g^i
    G[i] = s;
  }
  build_record<Q>(a.J[c], a.ginv + c * NS, G, K, a.tau, rec);
  // F at rest (rho = 1, U = 0), the start value of the chord iteration
  {
    double gd[NS], U0[D], N[Q], Np[Q];
    for (int i = 0; i < NS; i++) gd[i] = 2.0 * rec[L::GH + i];
    for (int i = 0; i < D; i++) U0[i] = 0.0;
    EqParts<Q, double> e;
    eq_parts<Q, double>(gd, U0, U0, e);
    for (int av = 0; av < Q; av++) {
      const int p = av <= H ? av : av - H;
      N[av] = rec[L::J] * lat_w<Q, double>(av) * eq_even<Q, double>(e, p);
    }
    CollideState<Q, double> cs;
    // chord iteration from F = 0 (the record's FR is still zero here)
    collide_cell<Q, double, false>(N, rec, 0.0, 1.0 / a.tau, 1e-15, 400, Np, cs);
    for (int i = 0; i < D; i++) rec[L::FR + i] = cs.conv ? cs.F[i] : 0.0;
  }
  // the local rest state for the final pass: deviations from the uniform
  // reference, their sum over all directions, and the rest weights
  {
    double gd[NS], U0[D], rsum = 0.0;
    for (int i = 0; i < NS; i++) gd[i] = 2.0 * rec[L::GH + i];
    for (int i = 0; i < D; i++) U0[i] = 0.0;
    EqParts<Q, double> e;
    eq_parts<Q, double>(gd, U0, U0, e);
    for (int p = 0; p <= H; p++) {
      const double rwp = lat_w<Q, double>(p) * eq_even<Q, double>(e, p);
      const double r = a.J[c] * rwp - lat_w<Q, double>(p) * a.nref;
      rec[L::RR + p] = r;
      rec[L::RW + p] = rwp;
      rsum += p == 0 ? r : 2.0 * r;
    }
    rec[L::RR + H + 1] = rsum;
  }
  // 16-bit storage relative to the rest state of Eq. 33 at the column that
  // holds each location (the fastest axis never changes the column, so only
  // the other axes decide a wall crossing): the constants and the per-link
  // column differences that let the collision work on N_a - o_a(own)
  if (a.ref_rest) {
    const Addr<Q> ad0(a.g, c);
    double own[Q], osum = 0.0;
    for (int av = 0; av < Q; av++) {
      own[av] = rest_ref<Q>(a.J[c], a.ginv + c * NS, av);
      osum += own[av];
    }
    rec[L::MDV] = osum - a.nref;   // the weights sum to one
    rec[L::MNV] = osum - a.J[c];
    for (int i = 0; i < D; i++) {
      double s = 0.0;
      for (int p = 1; p <= H; p++) s += rec[L::mp(p, i)] * 2.0 * (own[p] - lat_w<Q, double>(p) * a.nref);
      rec[L::SR + i] = s;
    }
    for (int av = 0; av < Q; av++) {
      for (int sg = -1; sg <= 1; sg += 2) {
        bool crs = false;
        for (int ax = 0; ax < D - 1; ax++) {
          const int cd = sg * Lat<Q>::c(av, ax);
          if ((cd > 0 && ad0.hi[ax]) || (cd < 0 && ad0.lo[ax])) crs = true;
        }
        const int64_t cb = crs || av == 0 ? c : (ad0.nb(av, sg) / a.nfast) * a.nfast;
        const double ob = rest_ref<Q>(a.J[cb], a.ginv + cb * NS, av);
        if (sg < 0)
          rec[L::DIN + av] = ob - own[av];
        else
          rec[L::DOUT + av] = own[av] - ob;
      }
    }
  }
  // a per-cell record ends at RR (see CoefLayout::stride)
  R *out = coef + r * a.stride;
  for (int k = 0; k < a.stride; k++) out[k] = k < L::NC ? static_cast<R>(rec[k]) : R(0);
  // reference-state part of J F as a hi/lo pair
  for (int i = 0; i < D; i++) {
    const R hi = static_cast<R>(rec[L::KW + i]);
    out[L::KW + i] = hi;
    out[L::KWL + i] = static_cast<R>(rec[L::KW + i] - static_cast<double>(hi));
  }
  // wall velocity: rigid motion of the adjacent wall, at the point halfway to the ghost node
  const Addr<Q> ad(a.g, c);
  double uw[3] = {0.0, 0.0, 0.0};
  for (int ax = 0; ax < D; ax++) {
    if (!(ad.lo[ax] || ad.hi[ax])) continue;
    const int side = ad.lo[ax] ? 0 : 1;
    int64_t q[3] = {ad.ic[0], ad.ic[1], ad.ic[2]}, gq[3] = {ad.ic[0], ad.ic[1], ad.ic[2]};
    gq[ax] += side ? 1 : -1;
    double x0[3], xg[3], xw[3], u[3];
    position(a.md, q, x0);
    position(a.md, gq, xg);
    for (int d = 0; d < 3; d++) xw[d] = 0.5 * (x0[d] + xg[d]);
    const double *om = a.wall_omega[ax][side];
    u[0] = om[1] * xw[2] - om[2] * xw[1];
    u[1] = om[2] * xw[0] - om[0] * xw[2];
    u[2] = om[0] * xw[1] - om[1] * xw[0];
    for (int d = 0; d < 3; d++) u[d] += a.wall_u[ax][side][d];
    for (int i = 0; i < D; i++) {
      double s = 0.0;
      for (int d = 0; d < D; d++) s += u[d] * a.gu[(c * D + i) * D + d];
      uw[i] = s;
    }
    break;
  }
  for (int i = 0; i < D; i++) out[L::UW + i] = static_cast<R>(uw[i]);
}

template <int Q>
static cudaError_t pack_q(const vlb_sim *sim, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  PackArgs a;
  a.md = m->md;
  a.g = make_grid(m);
  a.J = m->d_J;
  a.gu = m->d_gu;
  a.ginv = m->d_ginv;
  a.K = m->d_K;
  a.nrec = sim->ncoef;
  a.stride = sim->nc;
  a.nfast = m->md.n[m->md.dim - 1];
  a.plane = sim->plane;
  a.tau = sim->p.tau;
  a.ref_rest = sim->ref_rest;
  a.nref = sim->nref;
  for (int d = 0; d < 3; d++) a.body[d] = sim->p.body_force[d];
  for (int ax = 0; ax < 3; ax++)
    for (int sd = 0; sd < 2; sd++)
      for (int d = 0; d < 3; d++) {
        a.wall_u[ax][sd][d] = sim->p.wall_u[ax][sd][d];
        a.wall_omega[ax][sd][d] = sim->p.wall_omega[ax][sd][d];
      }
  const int threads = 128;
  const int64_t blocks = (a.nrec + threads - 1) / threads;
  if (arith_f64(sim->p.precision))
    k_pack_coef<Q, double><<<(unsigned)blocks, threads, 0, s>>>(a, (double *)sim->d_coef);
  else
    k_pack_coef<Q, float><<<(unsigned)blocks, threads, 0, s>>>(a, (float *)sim->d_coef);
  return cudaGetLastError();
}

cudaError_t launch_pack_coef(const vlb_sim *sim, cudaStream_t s) {
  return sim->mesh->md.q == 9 ? pack_q<9>(sim, s) : pack_q<19>(sim, s);
}

// ------------------------------------------------------------------ initial state
// N_a = J f^eq_a(rho, U, U~ = U), U^i = u . g^i (Eqs. 14, 33), normal layout
template <int Q, typename S>
__global__ void k_init(const double *J, const double *gu, const double *ginv, const double *rho,
                       const double *u, int64_t ncell, RefCtx ref, S *f) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2, H = Lat<Q>::H;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double U[D], gd[NS], zero[D];
  for (int i = 0; i < D; i++) {
    double s = 0.0;
    for (int d = 0; d < D; d++) s += u[c * D + d] * gu[(c * D + i) * D + d];
    U[i] = s;
    zero[i] = 0.0;
  }
  for (int i = 0; i < NS; i++) gd[i] = ginv[c * NS + i];
  for (int i = 0; i < D; i++) gd[sym<D>(i, i)] -= 1.0;
  EqParts<Q, double> e;
  eq_parts<Q, double>(gd, U, zero, e);
  const double r = rho[c], Jc = J[c];
  // stored relative to the storage reference of each location
  f[c] = store_s<S>(Jc * r * lat_w<Q, double>(0) * eq_even<Q, double>(e, 0) - ref_at<Q>(ref, 0, c));
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const double E = eq_even<Q, double>(e, p), O = eq_odd<Q, double>(e, U, p);
    const double w = lat_w<Q, double>(p), rw = Jc * r * w;
    f[p * ncell + c] = store_s<S>(rw * (E + O) - ref_at<Q>(ref, p, c));
    f[(p + H) * ncell + c] = store_s<S>(rw * (E - O) - ref_at<Q>(ref, p + H, c));
  }
}

// The same initial state for FP32 arithmetic (FP32 or 16-bit storage relative
// to the uniform reference n_ref): with J f^eq_a = J rho w_a (1 + x_a),
//   N_a - w_a n_ref = w_a [(J rho - n_ref) + J rho x_a],
// J rho - n_ref is formed in FP64 (one difference of large terms) and the
// bracket x_a in FP32, so every FP32 term is of the size of the deviation.
// (GB300's FP64 rate is a small fraction of its FP32 rate; the FP64 form of
// k_init is bound by it.)
template <int Q>
__device__ __forceinline__ float eq_even_x(const EqParts<Q, float> &e, int a) {
  constexpr int D = Lat<Q>::D;
  float cbc = 0.0f;
#pragma unroll
  for (int i = 0; i < D; i++) {
    const int ci = Lat<Q>::c(a, i);
    if (ci == 0) continue;
#pragma unroll
    for (int j = 0; j < D; j++) {
      const int cj = Lat<Q>::c(a, j);
      if (cj == 0) continue;
      if (ci * cj > 0)
        cbc += e.B[i][j];
      else
        cbc -= e.B[i][j];
    }
  }
  return (3.0f * cbc - e.trB) * 1.5f;
}

template <int Q, typename S>
__global__ void k_init_f32(const double *J, const double *gu, const double *ginv, const double *rho,
                           const double *u, int64_t ncell, double nref, S *f) {
  constexpr int D = Lat<Q>::D, NS = D * (D + 1) / 2, H = Lat<Q>::H;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  float U[D], gd[NS], zero[D];
  for (int i = 0; i < D; i++) {
    float s = 0.0f;
    for (int d = 0; d < D; d++) s = fmaf((float)u[c * D + d], (float)gu[(c * D + i) * D + d], s);
    U[i] = s;
    zero[i] = 0.0f;
  }
  // g^ii - 1 formed in FP64 before rounding
  for (int i = 0; i < D; i++)
    for (int j = i; j < D; j++)
      gd[sym<D>(i, j)] = (float)(ginv[c * NS + sym<D>(i, j)] - (i == j ? 1.0 : 0.0));
  EqParts<Q, float> e;
  eq_parts<Q, float>(gd, U, zero, e);
  const double jr = J[c] * rho[c];
  const float md = (float)(jr - nref), jrf = (float)jr;
  f[c] = store_s<S>(lat_w<Q, float>(0) * fmaf(jrf, eq_even_x<Q>(e, 0), md));
#pragma unroll
  for (int p = 1; p <= H; p++) {
    const float xe = eq_even_x<Q>(e, p), xo = eq_odd<Q, float>(e, U, p), w = lat_w<Q, float>(p);
    f[p * ncell + c] = store_s<S>(w * fmaf(jrf, xe + xo, md));
    f[(p + H) * ncell + c] = store_s<S>(w * fmaf(jrf, xe - xo, md));
  }
}

cudaError_t launch_init(const vlb_sim *sim, const double *d_rho, const double *d_u, cudaStream_t s) {
  const vlb_mesh *m = sim->mesh;
  const int threads = 128;
  const int64_t blocks = (m->ncell + threads - 1) / threads;
  const RefCtx ref = make_ref(sim);
  return with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    if constexpr (!std::is_same<S, double>::value) {
      // FP32 arithmetic for the uniform reference (the rest reference of
      // 16-bit storage keeps the FP64 form)
      if (!ref.rest) {
        if (m->md.q == 9)
          k_init_f32<9, S><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_gu, m->d_ginv, d_rho, d_u, m->ncell,
                                                                ref.nref, (S *)sim->d_f);
        else
          k_init_f32<19, S><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_gu, m->d_ginv, d_rho, d_u, m->ncell,
                                                                 ref.nref, (S *)sim->d_f);
        return cudaGetLastError();
      }
    }
    if (m->md.q == 9)
      k_init<9, S><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_gu, m->d_ginv, d_rho, d_u, m->ncell,
                                                        ref, (S *)sim->d_f);
    else
      k_init<19, S><<<(unsigned)blocks, threads, 0, s>>>(m->d_J, m->d_gu, m->d_ginv, d_rho, d_u, m->ncell,
                                                         ref, (S *)sim->d_f);
    return cudaGetLastError();
  });
}

}  // namespace vlb

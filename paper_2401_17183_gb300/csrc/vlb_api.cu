// vlb_api.cu -- host implementation of the C-ABI in include/vlb.h: argument
// validation, device memory ownership, launch sequencing and error reporting.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "vlb_internal.cuh"
#include "vlb_q39.cuh"

namespace {

// The packed FP32 arithmetic of the step kernel loads coefficient pairs as
// 8-byte values and quads as 16-byte values: every pair must start on an even
// element and every quad on a multiple of four of a record whose stride keeps
// 16-byte alignment.
template <int Q>
constexpr bool record_pairs_aligned() {
  using L = vlb::CoefLayout<Q>;
  constexpr int D = L::D;
  bool ok = L::template stride<float, true>() % 4 == 0 && L::template stride<float, false>() % 4 == 0 &&
            L::SREST % 4 == 0 && L::MPD % 4 == 0 && L::UW + D <= L::RR &&
            L::QM % 4 == 0 && L::HM % 2 == 0;
  // 16-byte quads of the link coefficients, 8-byte component-2 pairs
  for (int p = 1; p <= L::H; p++) ok = ok && L::mp(p, 0) % 4 == 0 && (D == 2 || L::mp(p, 2) % 2 == 0);
  // rows 0 and 1 of the chord step as 16-byte quads, row 2 likewise
  ok = ok && (2 * L::NQ) % 2 == 0 && (D == 2 || (L::row(L::QM, L::NQ, 2, 0) % 4 == 0 && L::NQ % 4 == 0));
  for (int k = 0; k < D; k++) ok = ok && L::row(L::HM, D, 0, k) % 2 == 0;
  return ok;
}
static_assert(record_pairs_aligned<9>() && record_pairs_aligned<19>(), "coefficient pairs must be 8-byte aligned");

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? VLB_ENOMEM : VLB_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
  } while (0)

int check_kernel_flags(int *d_err, cudaStream_t s) {
  int h = 0;
  CU(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (h & vlb::ERR_GEOM) return fail(VLB_EGEOM, "degenerate mesh cell (J <= 0 or D_i = D_-i)");
  if (h & vlb::ERR_NOCONV)
    return fail(VLB_ENOCONV, "local fixed-point solve for F hit its iteration cap");
  if (h & vlb::ERR_NONFINITE) return fail(VLB_ENONFINITE, "non-finite moment");
  return VLB_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

int ensure_io(vlb_sim *s, size_t bytes) {
  if (s->io_bytes >= bytes) return VLB_OK;
  dfree(s->d_io);
  s->io_bytes = 0;
  CU(cudaMalloc(&s->d_io, bytes));
  s->io_bytes = bytes;
  return VLB_OK;
}

}  // namespace

int vlb::set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

extern "C" {

const char *vlb_last_error(void) { return g_err; }

int vlb_lattice(int32_t lattice, int32_t *c, double *w) {
  if (lattice != VLB_D2Q9 && lattice != VLB_D3Q19 && lattice != VLB_D3Q39)
    return fail(VLB_EINVAL, "unknown lattice %d", lattice);
  for (int a = 0; a < lattice; a++) {
    for (int d = 0; d < 3; d++) {
      const int v = lattice == 9    ? vlb::Lat<9>::c(a, d)
                    : lattice == 19 ? vlb::Lat<19>::c(a, d)
                                    : vlb::Lat<39>::c(a, d);
      if (c) c[3 * a + d] = v;
    }
    if (w)
      w[a] = lattice == 9 ? vlb::lat_w<9, double>(a) : lattice == 19 ? vlb::lat_w<19, double>(a) : vlb::q39_w(a);
  }
  return VLB_OK;
}

int vlb_mesh_create(const vlb_mesh_desc *desc, vlb_mesh **out) {
  if (!out) return fail(VLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!desc || !desc->x) return fail(VLB_EINVAL, "desc or desc->x is NULL");
  const int dim = desc->dim, q = desc->lattice;
  if (!((dim == 2 && q == VLB_D2Q9) || (dim == 3 && (q == VLB_D3Q19 || q == VLB_D3Q39))))
    return fail(VLB_EINVAL, "dim %d with lattice %d is not supported (D2Q9 in 2D, D3Q19 or D3Q39 in 3D)", dim, q);
  if (q == VLB_D3Q39)
    for (int a = 0; a < 3; a++) {
      if (desc->bc[a] != VLB_PERIODIC || desc->n[a] < 3)
        return fail(VLB_EINVAL, "D3Q39 needs periodic axes of at least 3 cells (axis %d)", a);
      for (int k = 0; k < 9; k++)
        if (desc->period_rot[a][k] != 0.0) return fail(VLB_EINVAL, "D3Q39 takes no periodic rotations");
    }
  if (dim == 2 && desc->n[2] != 1) return fail(VLB_EINVAL, "n[2] must be 1 in 2D");
  for (int a = 0; a < dim; a++) {
    if (desc->n[a] < 1) return fail(VLB_EINVAL, "n[%d] = %lld < 1", a, (long long)desc->n[a]);
    if (desc->bc[a] != VLB_PERIODIC && desc->bc[a] != VLB_WALL)
      return fail(VLB_EINVAL, "bc[%d] = %d is not VLB_PERIODIC or VLB_WALL", a, desc->bc[a]);
    if (desc->bc[a] == VLB_WALL && desc->n[a] < 2)
      return fail(VLB_EINVAL, "a wall axis needs at least 2 nodes (axis %d)", a);
  }
  vlb_mesh *m = new (std::nothrow) vlb_mesh();
  if (!m) return fail(VLB_ENOMEM, "host allocation");
  vlb::MeshDev &md = m->md;
  md.dim = dim;
  md.q = q;
  for (int a = 0; a < 3; a++) {
    md.n[a] = a < dim ? desc->n[a] : 1;
    md.bc[a] = a < dim ? desc->bc[a] : VLB_PERIODIC;
    md.has_rot[a] = 0;
    for (int d = 0; d < 3; d++) md.shift[a][d] = desc->period_shift[a][d];
    for (int k = 0; k < 9; k++) {
      md.rot[a][k] = desc->period_rot[a][k];
      if (md.rot[a][k] != 0.0) md.has_rot[a] = 1;
    }
  }
  md.dx = desc->dx > 0.0 ? desc->dx : 1.0;
  if (desc->wall_links != VLB_WALL_LINKS_ZERO && desc->wall_links != VLB_WALL_LINKS_GHOST) {
    delete m;
    return fail(VLB_EINVAL, "wall_links = %d is not ZERO or GHOST", desc->wall_links);
  }
  md.wall_links = desc->wall_links;
  m->ncell = md.n[0] * md.n[1] * md.n[2];
  cudaGetDevice(&m->device);
  const int64_t nc = m->ncell;
  const int NS = dim * (dim + 1) / 2;
  int rc = VLB_OK;
  int *d_flag = nullptr;
  double *d_part = nullptr;
  auto cleanup = [&](int code) {
    dfree(d_flag);
    dfree(d_part);
    if (code != VLB_OK) {
      vlb_mesh_destroy(m);
      m = nullptr;
    }
    return code;
  };
  {
    cudaError_t e = cudaMalloc(&m->d_x, sizeof(double) * nc * dim);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_J, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_gl, sizeof(double) * nc * dim * dim);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_gu, sizeof(double) * nc * dim * dim);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_ginv, sizeof(double) * nc * NS);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_K, sizeof(double) * nc * q * dim);
    if (e == cudaSuccess) e = cudaMalloc(&d_flag, sizeof(int) * 2);
    if (e != cudaSuccess)
      return cleanup(fail(VLB_ENOMEM, "mesh device allocation: %s", cudaGetErrorString(e)));
    e = cudaMemcpy(m->d_x, desc->x, sizeof(double) * nc * dim, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_flag, 0, sizeof(int) * 2);
    if (e != cudaSuccess) return cleanup(fail(VLB_ECUDA, "mesh upload: %s", cudaGetErrorString(e)));
  }
  md.x = m->d_x;
  cudaError_t e = vlb::launch_geometry(m, d_flag, 0);
  if (e != cudaSuccess) return cleanup(fail(VLB_ECUDA, "geometry launch: %s", cudaGetErrorString(e)));
  rc = check_kernel_flags(d_flag, 0);
  if (rc) return cleanup(rc);
  // diagnostics
  const int64_t nblk = std::min<int64_t>(1024, (nc + vlb::kStatThreads - 1) / vlb::kStatThreads);
  if (cudaMalloc(&d_part, sizeof(double) * 5 * nblk) != cudaSuccess)
    return cleanup(fail(VLB_ENOMEM, "stats scratch"));
  e = q == VLB_D3Q39 ? vlb::q39_mesh_stats(m, d_part, nblk, 0) : vlb::launch_mesh_stats(m, d_part, nblk, 0);
  if (e != cudaSuccess) return cleanup(fail(VLB_ECUDA, "stats launch: %s", cudaGetErrorString(e)));
  // D3Q39 keeps per-cell geometry (no plane records): report "varies"
  e = q == VLB_D3Q39 ? cudaMemset(d_flag + 1, 1, sizeof(int)) : vlb::launch_plane_check(m, d_flag + 1, 0);
  if (e != cudaSuccess) return cleanup(fail(VLB_ECUDA, "plane check: %s", cudaGetErrorString(e)));
  double *h = new (std::nothrow) double[5 * nblk];
  if (!h) return cleanup(fail(VLB_ENOMEM, "host stats"));
  int hflag = 0;
  e = cudaMemcpy(h, d_part, sizeof(double) * 5 * nblk, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&hflag, d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete[] h;
    return cleanup(fail(VLB_ECUDA, "stats download: %s", cudaGetErrorString(e)));
  }
  double v[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
  for (int64_t b = 0; b < nblk; b++)
    for (int k = 0; k < 5; k++) v[k] = std::min(v[k], h[b * 5 + k]);
  delete[] h;
  m->stats.J_min = v[0];
  m->stats.J_max = -v[1];
  m->stats.feq_rest_min = v[2];
  m->stats.ginv_diag_min = v[3];
  m->stats.ginv_diag_max = -v[4];
  m->stats.invariant_fast_axis = hflag ? 0 : 1;
  m->stats.ncell = nc;
  rc = cleanup(VLB_OK);
  *out = m;
  return rc;
}

int vlb_mesh_info(const vlb_mesh *mesh, vlb_mesh_stats *out) {
  if (!mesh || !out) return fail(VLB_EINVAL, "NULL argument");
  *out = mesh->stats;
  return VLB_OK;
}

int vlb_mesh_geometry(const vlb_mesh *m, double *J, double *g_low, double *ginv, double *K) {
  if (!m) return fail(VLB_EINVAL, "NULL mesh");
  const int dim = m->md.dim, q = m->md.q, NS = dim * (dim + 1) / 2;
  const int64_t nc = m->ncell;
  if (J) CU(cudaMemcpy(J, m->d_J, sizeof(double) * nc, cudaMemcpyDeviceToHost));
  if (g_low) CU(cudaMemcpy(g_low, m->d_gl, sizeof(double) * nc * dim * dim, cudaMemcpyDeviceToHost));
  if (K) CU(cudaMemcpy(K, m->d_K, sizeof(double) * nc * q * dim, cudaMemcpyDeviceToHost));
  if (ginv) {
    double *tmp = new (std::nothrow) double[nc * NS];
    if (!tmp) return fail(VLB_ENOMEM, "host buffer");
    cudaError_t e = cudaMemcpy(tmp, m->d_ginv, sizeof(double) * nc * NS, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      delete[] tmp;
      return fail(VLB_ECUDA, "ginv download: %s", cudaGetErrorString(e));
    }
    for (int64_t c = 0; c < nc; c++)
      for (int i = 0; i < dim; i++)
        for (int j = 0; j < dim; j++) {
          const int k = dim == 2 ? vlb::sym<2>(i, j) : vlb::sym<3>(i, j);
          ginv[(c * dim + i) * dim + j] = tmp[c * NS + k];
        }
    delete[] tmp;
  }
  return VLB_OK;
}

void vlb_mesh_destroy(vlb_mesh *m) {
  if (!m) return;
  dfree(m->d_x);
  dfree(m->d_J);
  dfree(m->d_gl);
  dfree(m->d_gu);
  dfree(m->d_ginv);
  dfree(m->d_K);
  delete m;
}

static int upload_fields(vlb_sim *s, const double *rho, const double *u) {
  const int64_t nc = s->mesh->ncell;
  const int dim = s->mesh->md.dim;
  int rc = ensure_io(s, sizeof(double) * nc * (1 + dim));
  if (rc) return rc;
  double *d_rho = s->d_io, *d_u = s->d_io + nc;
  CU(cudaMemcpyAsync(d_rho, rho, sizeof(double) * nc, cudaMemcpyHostToDevice, s->stream));
  CU(cudaMemcpyAsync(d_u, u, sizeof(double) * nc * dim, cudaMemcpyHostToDevice, s->stream));
  CU(s->mesh->md.q == VLB_D3Q39 ? vlb::q39_init(s, d_rho, d_u, s->stream)
                                 : vlb::launch_init(s, d_rho, d_u, s->stream));
  CU(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  s->t = 0;
  return VLB_OK;
}

int vlb_init(const vlb_mesh *mesh, const vlb_params *params, const double *rho, const double *u,
             vlb_sim **out) {
  if (!out) return fail(VLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !params || !rho || !u) return fail(VLB_EINVAL, "NULL argument");
  if (!(params->tau > 0.5)) return fail(VLB_EINVAL, "tau = %g must exceed 1/2", params->tau);
  if (params->precision < VLB_F64 || params->precision > VLB_BF16)
    return fail(VLB_EINVAL, "unknown precision %d", params->precision);
  if (params->reference != VLB_REF_UNIFORM && params->reference != VLB_REF_REST)
    return fail(VLB_EINVAL, "unknown reference %d", params->reference);
  if (params->coef_mode < VLB_COEF_AUTO || params->coef_mode > VLB_COEF_PLANE)
    return fail(VLB_EINVAL, "unknown coef_mode %d", params->coef_mode);
  const int dim = mesh->md.dim, q = mesh->md.q;
  if (q == VLB_D3Q39 && params->precision != VLB_F64)
    return fail(VLB_EINVAL, "D3Q39 runs in FP64 (precision VLB_F64)");
  if (q == VLB_D3Q39 && params->coef_mode == VLB_COEF_PLANE)
    return fail(VLB_EINVAL, "D3Q39 reads per-cell geometry (coef_mode AUTO or FULL)");
  bool moving = false;
  int nwall = 0;
  for (int a = 0; a < dim; a++) nwall += mesh->md.bc[a] == VLB_WALL;
  for (int a = 0; a < 3; a++)
    for (int sd = 0; sd < 2; sd++)
      for (int d = 0; d < 3; d++)
        if (params->wall_u[a][sd][d] != 0.0 || params->wall_omega[a][sd][d] != 0.0) moving = true;
  if (moving && nwall > 1)
    return fail(VLB_EINVAL, "moving walls need a single wall axis (corner cells would touch two walls)");
  vlb_sim *s = new (std::nothrow) vlb_sim();
  if (!s) return fail(VLB_ENOMEM, "host allocation");
  s->mesh = mesh;
  s->p = *params;
  if (s->p.max_iter <= 0) s->p.max_iter = 100;
  if (s->p.tol <= 0.0) s->p.tol = params->precision == VLB_F64 ? 1e-14 : 1e-6;
  s->stream = (cudaStream_t)params->stream;
  // uniform storage reference n_ref = rho_0 J_ref, rho_0 = 1, J_ref mid-range of J,
  // rounded to a value FP32 represents exactly, so that the FP32 step kernel
  // and the FP64 kernels (initialisation, moments, state) use the same one
  s->nref = (double)(float)(0.5 * (mesh->stats.J_min + mesh->stats.J_max));
  bool plane = false;
  if (params->coef_mode == VLB_COEF_PLANE) {
    if (!mesh->stats.invariant_fast_axis) {
      delete s;
      return fail(VLB_EINVAL, "coef_mode PLANE needs a geometry that does not vary along the fastest axis");
    }
    plane = true;
  } else if (params->coef_mode == VLB_COEF_AUTO) {
    plane = mesh->stats.invariant_fast_axis != 0 && mesh->md.n[dim - 1] > 1;
  }
  s->plane = plane ? 1 : 0;
  s->ncoef = plane ? mesh->ncell / mesh->md.n[dim - 1] : mesh->ncell;
  const bool f16 = params->precision == VLB_F16 || params->precision == VLB_BF16;
  if (params->reference == VLB_REF_REST && f16) {
    if (!plane) {
      delete s;
      return fail(VLB_EINVAL,
                  "reference REST needs plane mode (a geometry that does not vary along the fastest axis)");
    }
    s->ref_rest = 1;
  }
  const bool f64 = vlb::arith_f64(params->precision);
  using L9 = vlb::CoefLayout<9>;
  using L19 = vlb::CoefLayout<19>;
  s->nc = q == 9    ? (plane ? L9::stride<float, true>() : L9::stride<float, false>())
          : q == 19 ? (plane ? L19::stride<float, true>() : L19::stride<float, false>())
                    : 0;  // D3Q39: no records, the kernels read the mesh geometry
  if (q == VLB_D3Q39) {
    // D3Q39: no records; per cell the chord data of its force map (q39_prepare)
    s->nc = 12;
    s->ncoef = mesh->ncell;
  }
  const size_t es = f64 ? 8 : 4;
  // 16 bytes of padding: a 16-bit population is read as the aligned 32-bit
  // word that contains it
  cudaError_t e = cudaMalloc(&s->d_f, vlb::storage_bytes(params->precision) * q * mesh->ncell + 16);
  if (e == cudaSuccess && s->ncoef > 0) e = cudaMalloc(&s->d_coef, es * s->nc * s->ncoef);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_err, sizeof(int));
  if (e != cudaSuccess) {
    vlb_destroy(s);
    return fail(VLB_ENOMEM, "simulation device allocation: %s", cudaGetErrorString(e));
  }
  e = q == VLB_D3Q39 ? vlb::q39_prepare(s, s->stream) : vlb::launch_pack_coef(s, s->stream);
  if (e != cudaSuccess) {
    vlb_destroy(s);
    return fail(VLB_ECUDA, "coefficient pack: %s", cudaGetErrorString(e));
  }
  int rc = upload_fields(s, rho, u);
  if (rc == VLB_OK) rc = check_kernel_flags(s->d_err, s->stream);
  if (rc) {
    vlb_destroy(s);
    return rc;
  }
  *out = s;
  return VLB_OK;
}

int vlb_reset(vlb_sim *s, const double *rho, const double *u) {
  if (!s || !rho || !u) return fail(VLB_EINVAL, "NULL argument");
  int rc = upload_fields(s, rho, u);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream));
  return VLB_OK;
}

int vlb_step(vlb_sim *s, int64_t nsteps) {
  if (!s) return fail(VLB_EINVAL, "NULL sim");
  if (nsteps < 0) return fail(VLB_EINVAL, "nsteps < 0");
  for (int64_t k = 0; k < nsteps; k++) {
    cudaError_t e = s->mesh->md.q == VLB_D3Q39 ? vlb::q39_step(s, (int)(s->t & 1), s->stream)
                                               : vlb::launch_step(s, (int)(s->t & 1), s->stream);
    if (e != cudaSuccess) return fail(VLB_ECUDA, "step launch: %s", cudaGetErrorString(e));
    s->t++;
  }
  return VLB_OK;
}

int vlb_sync(vlb_sim *s) {
  if (!s) return fail(VLB_EINVAL, "NULL sim");
  return check_kernel_flags(s->d_err, s->stream);
}

int vlb_moments(vlb_sim *s, double *rho, double *u, double *u_tilde, double *totals) {
  if (!s) return fail(VLB_EINVAL, "NULL sim");
  const vlb_mesh *m = s->mesh;
  const int dim = m->md.dim;
  const int64_t nc = m->ncell;
  if (!s->d_fields) CU(cudaMalloc(&s->d_fields, sizeof(double) * nc * (1 + 2 * dim)));
  const int64_t nblk = std::min<int64_t>(4 * 152, (nc + vlb::kMomThreads - 1) / vlb::kMomThreads);
  if (!s->d_partial) {
    CU(cudaMalloc(&s->d_partial, sizeof(double) * 7 * 4 * 152));
    CU(cudaMalloc(&s->d_totals, sizeof(double) * 7));
  }
  if (m->md.q == VLB_D3Q39) {
    CU(vlb::q39_moments(s, s->d_fields, s->d_partial, nblk, s->stream));
    CU(vlb::launch_finish_totals(s->d_partial, nblk, s->d_totals, s->stream));
  } else {
    CU(vlb::launch_moments(s, s->d_fields, nblk, s->stream));
    CU(vlb::launch_totals(s, s->d_partial, 4 * 152, s->d_totals, s->stream));
  }
  int rc = check_kernel_flags(s->d_err, s->stream);
  if (rc) return rc;
  // the kernel writes rho [nc], u [nc][dim] and u~ [nc][dim] one after the
  // other: one contiguous copy each, straight into the caller's arrays, in
  // the simulation's stream, then one wait for all of them
  double t7[7];
  if (totals) CU(cudaMemcpyAsync(t7, s->d_totals, sizeof(t7), cudaMemcpyDeviceToHost, s->stream));
  if (rho) CU(cudaMemcpyAsync(rho, s->d_fields, sizeof(double) * nc, cudaMemcpyDeviceToHost, s->stream));
  if (u) CU(cudaMemcpyAsync(u, s->d_fields + nc, sizeof(double) * nc * dim, cudaMemcpyDeviceToHost, s->stream));
  if (u_tilde)
    CU(cudaMemcpyAsync(u_tilde, s->d_fields + nc * (1 + dim), sizeof(double) * nc * dim, cudaMemcpyDeviceToHost,
                       s->stream));
  CU(cudaStreamSynchronize(s->stream));
  if (totals) {
    for (int k = 0; k < 7; k++) totals[k] = 0.0;
    totals[0] = t7[0];
    for (int d = 0; d < dim; d++) {
      totals[1 + d] = t7[1 + d];
      totals[4 + d] = t7[4 + d];
    }
  }
  return VLB_OK;
}

int vlb_get_state(vlb_sim *s, double *N) {
  if (!s || !N) return fail(VLB_EINVAL, "NULL argument");
  const int64_t nc = s->mesh->ncell;
  const int q = s->mesh->md.q;
  int rc = ensure_io(s, sizeof(double) * nc * q);
  if (rc) return rc;
  CU(q == VLB_D3Q39 ? vlb::q39_get_state(s, s->d_io, s->stream) : vlb::launch_get_state(s, s->d_io, s->stream));
  rc = check_kernel_flags(s->d_err, s->stream);
  if (rc) return rc;
  CU(cudaMemcpy(N, s->d_io, sizeof(double) * nc * q, cudaMemcpyDeviceToHost));
  return VLB_OK;
}

int vlb_set_state(vlb_sim *s, const double *N) {
  if (!s || !N) return fail(VLB_EINVAL, "NULL argument");
  const int64_t nc = s->mesh->ncell;
  const int q = s->mesh->md.q;
  int rc = ensure_io(s, sizeof(double) * nc * q);
  if (rc) return rc;
  CU(cudaMemcpyAsync(s->d_io, N, sizeof(double) * nc * q, cudaMemcpyHostToDevice, s->stream));
  CU(q == VLB_D3Q39 ? vlb::q39_set_state(s, s->d_io, s->stream) : vlb::launch_set_state(s, s->d_io, s->stream));
  CU(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  CU(cudaStreamSynchronize(s->stream));
  s->t = 0;
  return VLB_OK;
}

int64_t vlb_time(const vlb_sim *s) { return s ? s->t : -1; }

int vlb_sim_layout(const vlb_sim *s, int32_t *coef_per_cell, int32_t *plane_mode, int64_t *records) {
  if (!s) return fail(VLB_EINVAL, "NULL sim");
  if (coef_per_cell) *coef_per_cell = s->nc;
  if (plane_mode) *plane_mode = s->plane;
  if (records) *records = s->ncoef;
  return VLB_OK;
}

void vlb_destroy(vlb_sim *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  dfree(s->d_f);
  dfree(s->d_coef);
  dfree(s->d_err);
  dfree(s->d_fields);
  dfree(s->d_partial);
  dfree(s->d_totals);
  dfree(s->d_io);
  delete s;
}

}  // extern "C"

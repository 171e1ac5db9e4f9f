// vlb_noalloc.cu -- vlb_totals_noalloc: the conservation totals of
// vlb_moments (mass, P, M), computed without allocating any memory.
//
// Some callers cannot call cudaMalloc: code whose device memory comes from a
// fixed budget or from a pool allocator it does not own, and latency-bound
// monitoring loops in which an allocation (which can synchronise the device)
// is not acceptable. vlb_moments allocates its staging buffers on first use;
// this variant instead reduces into a file-scope device array whose size is
// fixed when the library is built, and writes the result to device memory
// the caller provides.
#include <mutex>

#include "vlb_addr.cuh"

namespace vlb {
namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNaCellsPerBlock = 16384;  // 64 cells per thread
constexpr int kNaMaxBlocks = 4096;           // so at most 67,108,864 cells
constexpr int kNaTotals = 7;

// Block partial sums, 4096 x 7 doubles (224 KiB) on every device that loads
// the library, for as long as the process runs. Every call overwrites the
// slots it reads (one per block it launches), so nothing needs clearing
// between calls; two calls that overlap on the GPU share this array and race.
static __device__ __align__(256) double g_totals_scratch[kNaMaxBlocks * kNaTotals];

struct TotArgs {
  const void *f;
  Grid g;
  int64_t ncell;
  int64_t per_block;
  const double *gl;
  RefCtx ref;
  double rot[3][9];
  int32_t has_rot[3];
  int32_t periodic[3];
};

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void na_block_sum(double (&v)[kNaTotals], double *out) {
  __shared__ double sh[kNaTotals][kNaThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNaTotals; k++) {
    const double s = na_warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kNaTotals; k++) {
      double s = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
      s = na_warp_sum(s);
      if (lane == 0) out[k] = s;
    }
  }
}

// block b sums cells [b * per_block, (b + 1) * per_block): mass = sum N,
// P = sum e_a(q) N_a, M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a
template <int Q, typename S, bool ODD>
__global__ void __launch_bounds__(kNaThreads) k_totals_noalloc(const TotArgs a, double *scratch) {
  constexpr int D = Lat<Q>::D;
  const S *f = static_cast<const S *>(a.f);
  double acc[kNaTotals] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t c0 = (int64_t)blockIdx.x * a.per_block;
  const int64_t c1 = c0 + a.per_block < a.ncell ? c0 + a.per_block : a.ncell;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const Addr<Q> ad(a.g, c);
    double N[Q];
    pull_abs<Q, ODD, S>(f, a.ncell, ad, a.ref, N);
    double gl[D][D];
    for (int i = 0; i < D; i++)
      for (int d = 0; d < D; d++) gl[i][d] = a.gl[(c * D + i) * D + d];
#pragma unroll 1
    for (int av = 0; av < Q; av++) {
      const double n = N[av];
      double e[D], eb[D];
      for (int d = 0; d < D; d++) {
        double s = 0.0;
        for (int i = 0; i < D; i++) s += Lat<Q>::c(av, i) * gl[i][d];
        e[d] = s;
        eb[d] = s;
      }
      if (av != 0 && !ad.crosses(av, -1)) {
        const int64_t nb = ad.nb(av, -1);
        double gn[D][D];
        for (int i = 0; i < D; i++)
          for (int d = 0; d < D; d++) gn[i][d] = a.gl[(nb * D + i) * D + d];
        for (int ax = 0; ax < D; ax++) {
          const int cax = Lat<Q>::c(av, ax);
          if (!a.has_rot[ax] || !a.periodic[ax] || cax == 0) continue;
          const bool below = (cax > 0 && ad.ic[ax] == 0);
          const bool above = (cax < 0 && ad.ic[ax] == a.g.n[ax] - 1);
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
      acc[0] += n;
      for (int d = 0; d < D; d++) {
        acc[1 + d] += e[d] * n;
        acc[4 + d] += 0.5 * (e[d] + eb[d]) * n;
      }
    }
  }
  na_block_sum(acc, scratch + (int64_t)blockIdx.x * kNaTotals);
}

// fixed-order sum of the block partials into the caller's 7 doubles
__global__ void __launch_bounds__(kNaThreads) k_totals_noalloc_finish(const double *scratch,
                                                                      int64_t nblk, double *out) {
  double v[kNaTotals] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int k = 0; k < kNaTotals; k++) v[k] += scratch[b * kNaTotals + k];
  na_block_sum(v, out);
}

// device address of g_totals_scratch, looked up once per device
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
double *g_na_addr[kNaMaxDevices] = {};

cudaError_t scratch_address(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_addr[dev]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_totals_scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

template <int Q, typename S>
cudaError_t launch_na(const vlb_sim *sim, double *scratch, int64_t nblk, double *d_out) {
  const vlb_mesh *m = sim->mesh;
  TotArgs a;
  a.f = sim->d_f;
  a.g = make_grid(m);
  a.ncell = m->ncell;
  a.per_block = kNaCellsPerBlock;
  a.gl = m->d_gl;
  a.ref = make_ref(sim);
  for (int d = 0; d < 3; d++) {
    a.has_rot[d] = m->md.has_rot[d];
    a.periodic[d] = (d < m->md.dim && m->md.bc[d] == VLB_PERIODIC) ? 1 : 0;
    for (int k = 0; k < 9; k++) a.rot[d][k] = m->md.rot[d][k];
  }
  if (sim->t & 1)
    k_totals_noalloc<Q, S, true><<<(unsigned)nblk, kNaThreads, 0, sim->stream>>>(a, scratch);
  else
    k_totals_noalloc<Q, S, false><<<(unsigned)nblk, kNaThreads, 0, sim->stream>>>(a, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_totals_noalloc_finish<<<1, kNaThreads, 0, sim->stream>>>(scratch, nblk, d_out);
  return cudaGetLastError();
}

}  // namespace
}  // namespace vlb

extern "C" int vlb_totals_noalloc(vlb_sim *sim, double *d_totals) {
  if (!sim || !d_totals) return vlb::set_error(VLB_EINVAL, "vlb_totals_noalloc: NULL argument");
  const vlb_mesh *m = sim->mesh;
  if (m->md.q != VLB_D2Q9 && m->md.q != VLB_D3Q19)
    return vlb::set_error(VLB_EINVAL, "vlb_totals_noalloc: D2Q9 and D3Q19 only; use vlb_moments");
  const int64_t nblk = (m->ncell + vlb::kNaCellsPerBlock - 1) / vlb::kNaCellsPerBlock;
  if (nblk > vlb::kNaMaxBlocks)
    return vlb::set_error(VLB_EINVAL,
                          "vlb_totals_noalloc: %lld cells exceed the fixed scratch of %d blocks x "
                          "%lld cells = %lld cells; use vlb_moments",
                          (long long)m->ncell, vlb::kNaMaxBlocks, (long long)vlb::kNaCellsPerBlock,
                          (long long)vlb::kNaMaxBlocks * vlb::kNaCellsPerBlock);
  if (m->device < 0 || m->device >= vlb::kNaMaxDevices)
    return vlb::set_error(VLB_EINVAL, "vlb_totals_noalloc: device %d out of range", m->device);
  double *scratch = nullptr;
  cudaError_t e = vlb::scratch_address(m->device, &scratch);
  if (e != cudaSuccess)
    return vlb::set_error(VLB_ECUDA, "vlb_totals_noalloc: cudaGetSymbolAddress: %s",
                          cudaGetErrorString(e));
  e = vlb::with_storage(sim->p.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return m->md.q == 9 ? vlb::launch_na<9, S>(sim, scratch, nblk, d_totals)
                        : vlb::launch_na<19, S>(sim, scratch, nblk, d_totals);
  });
  if (e != cudaSuccess)
    return vlb::set_error(VLB_ECUDA, "vlb_totals_noalloc: launch: %s", cudaGetErrorString(e));
  return VLB_OK;
}

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

constexpr int64_t kNaCellsPerBlock = 16384;  // the documented size limit: 4096 x 16384 cells
constexpr int kNaMaxBlocks = 4096;           // block partial sums the scratch holds
constexpr int kNaTotals = 7;

// Block partial sums, 4096 x 7 doubles (224 KiB) on every device that loads
// the library, for as long as the process runs. Every call overwrites the
// slots it reads (one per block it launches), so nothing needs clearing
// between calls; two calls that overlap on the GPU share this array and race.
static __device__ __align__(256) double g_totals_scratch[kNaMaxBlocks * kNaTotals];

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
  // the kernels run on the mesh's device, whatever device the calling thread
  // has current (the scratch address belongs to that device)
  int cur = 0;
  e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != m->device) e = cudaSetDevice(m->device);
  if (e != cudaSuccess)
    return vlb::set_error(VLB_ECUDA, "vlb_totals_noalloc: device: %s", cudaGetErrorString(e));
  // the same totals kernels as vlb_moments, with the fixed array as the
  // per-block partial sums (at most kNaMaxBlocks blocks; each loops over as
  // many cells or columns as it needs)
  e = vlb::launch_totals(sim, scratch, vlb::kNaMaxBlocks, d_totals, sim->stream);
  if (cur != m->device) cudaSetDevice(cur);
  if (e != cudaSuccess)
    return vlb::set_error(VLB_ECUDA, "vlb_totals_noalloc: launch: %s", cudaGetErrorString(e));
  return VLB_OK;
}

// vlb_batch.cu -- many simulations advanced by one kernel launch per time step.
//
// Each member's tiles are cut into runs of `run` tiles; every run is one block
// of a single launch of k_step_batch, which reads its member's kernel
// arguments from a device array. The per-cell work is that of vlb_step, so a
// batch reproduces the members' individual steps bit for bit. Whole runs of
// 32 steps replay a CUDA graph of 32 kernel nodes (alternating A-A parity).
#include <new>

#include "vlb_step.cuh"

namespace vlb {
namespace {

constexpr int kGraphSteps = 32;

using BatchKernel = void (*)(const StepArgs *, const BatchItem *);

struct BatchKind {
  int q;
  bool f64;
  bool plane;
};

template <int Q, typename R, bool PLANE>
BatchKernel pick_kernel(bool odd) {
  return odd ? k_step_batch<Q, R, R, true, PLANE, int32_t> : k_step_batch<Q, R, R, false, PLANE, int32_t>;
}

BatchKernel batch_kernel(const BatchKind &k, bool odd) {
  if (k.q == 9) {
    if (k.f64) return k.plane ? pick_kernel<9, double, true>(odd) : pick_kernel<9, double, false>(odd);
    return k.plane ? pick_kernel<9, float, true>(odd) : pick_kernel<9, float, false>(odd);
  }
  if (k.f64) return k.plane ? pick_kernel<19, double, true>(odd) : pick_kernel<19, double, false>(odd);
  return k.plane ? pick_kernel<19, float, true>(odd) : pick_kernel<19, float, false>(odd);
}

size_t batch_smem(const BatchKind &k) {
  if (k.q == 9)
    return k.f64 ? sizeof(StepSmem<9, double, double>) : sizeof(StepSmem<9, float, float>);
  return k.f64 ? sizeof(StepSmem<19, double, double>) : sizeof(StepSmem<19, float, float>);
}

BatchKind kind_of(const vlb_batch *b) {
  const vlb_sim *s = b->sims[0];
  return BatchKind{s->mesh->md.q, s->p.precision == VLB_F64, s->plane != 0};
}

int64_t member_tiles(const vlb_sim *s) {
  const vlb_mesh *m = s->mesh;
  const int dim = m->md.dim;
  const int64_t nfast = m->md.n[dim - 1];
  const int64_t ntf = (nfast + kStepThreads - 1) / kStepThreads;
  return ntf * (dim == 3 ? m->md.n[0] * m->md.n[1] : m->md.n[0]);
}

int64_t total_tiles(const vlb_batch *b) {
  int64_t t = 0;
  for (const vlb_sim *s : b->sims) t += member_tiles(s);
  return t;
}

// blocks the batch kernel keeps resident on the device
int64_t batch_resident(const vlb_batch *b) {
  const BatchKind k = kind_of(b);
  return resident_blocks(reinterpret_cast<const void *>(batch_kernel(k, false)), batch_smem(k));
}

// cut every member into runs of `run` tiles and upload the work list
cudaError_t set_run(vlb_batch *b, int64_t run) {
  std::vector<BatchItem> items;
  for (size_t m = 0; m < b->sims.size(); m++) {
    const int64_t nt = member_tiles(b->sims[m]);
    for (int64_t t = 0; t < nt; t += run) {
      BatchItem it;
      it.sim = (int32_t)m;
      it.pad = 0;
      it.t0 = t;
      it.t1 = t + run < nt ? t + run : nt;
      items.push_back(it);
    }
  }
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size());
    if (e != cudaSuccess) return e;
    b->items_cap = items.size();
  }
  cudaError_t e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  b->run = run;
  b->nitems = (int64_t)items.size();
  return cudaSuccess;
}

cudaError_t launch_one(const vlb_batch *b, bool odd) {
  const BatchKind k = kind_of(b);
  const BatchKernel kern = batch_kernel(k, odd);
  kern<<<(unsigned)b->nitems, kStepThreads, batch_smem(k), b->stream>>>(
      static_cast<const StepArgs *>(b->d_args), static_cast<const BatchItem *>(b->d_items));
  return cudaGetLastError();
}

// kGraphSteps kernel nodes in a chain, even parity first
cudaError_t build_graph(vlb_batch *b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  const BatchKind k = kind_of(b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  const StepArgs *args = static_cast<const StepArgs *>(b->d_args);
  const BatchItem *items = static_cast<const BatchItem *>(b->d_items);
  void *params[2] = {(void *)&args, (void *)&items};
  cudaGraphNode_t prev = nullptr;
  for (int i = 0; i < kGraphSteps && e == cudaSuccess; i++) {
    cudaKernelNodeParams p = {};
    p.func = reinterpret_cast<void *>(batch_kernel(k, (i & 1) != 0));
    p.gridDim = dim3((unsigned)b->nitems);
    p.blockDim = dim3(kStepThreads);
    p.sharedMemBytes = (unsigned)batch_smem(k);
    p.kernelParams = params;
    cudaGraphNode_t node;
    e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
    prev = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) b->graph_run = b->run;
  return e;
}

cudaError_t run_steps(vlb_batch *b, int64_t n) {
  const int64_t start = b->sims[0]->t;
  int64_t t = start;
  cudaError_t e = cudaSuccess;
  if (n > 0 && (t & 1)) {
    e = launch_one(b, true);
    n--;
    t++;
  }
  if (e == cudaSuccess && n >= kGraphSteps && (!b->graph || b->graph_run != b->run)) e = build_graph(b);
  while (e == cudaSuccess && n >= kGraphSteps) {
    e = cudaGraphLaunch(b->graph, b->stream);
    n -= kGraphSteps;
    t += kGraphSteps;
  }
  while (e == cudaSuccess && n > 0) {
    e = launch_one(b, (t & 1) != 0);
    n--;
    t++;
  }
  for (vlb_sim *s : b->sims) s->t += t - start;
  return e;
}

}  // namespace
}  // namespace vlb

extern "C" {

int vlb_batch_create(vlb_sim *const *sims, int32_t nsims, vlb_batch **out) {
  if (!out) return vlb::set_error(VLB_EINVAL, "vlb_batch_create: out is NULL");
  *out = nullptr;
  if (!sims || nsims < 1) return vlb::set_error(VLB_EINVAL, "vlb_batch_create: no simulations");
  const vlb_sim *s0 = sims[0];
  if (!s0) return vlb::set_error(VLB_EINVAL, "vlb_batch_create: NULL simulation");
  if (s0->p.precision != VLB_F32 && s0->p.precision != VLB_F64)
    return vlb::set_error(VLB_EINVAL, "vlb_batch_create: batches take VLB_F32 or VLB_F64 members");
  if (s0->mesh->md.q != VLB_D2Q9 && s0->mesh->md.q != VLB_D3Q19)
    return vlb::set_error(VLB_EINVAL, "vlb_batch_create: batches take D2Q9 or D3Q19 members");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return vlb::set_error(VLB_ECUDA, "vlb_batch_create: no device");
  for (int32_t i = 0; i < nsims; i++) {
    const vlb_sim *s = sims[i];
    if (!s) return vlb::set_error(VLB_EINVAL, "vlb_batch_create: NULL simulation %d", i);
    const vlb_mesh *m = s->mesh;
    if (m->device != dev)
      return vlb::set_error(VLB_EINVAL, "vlb_batch_create: member %d lives on device %d, current is %d", i,
                            m->device, dev);
    if (m->md.q != s0->mesh->md.q || s->p.precision != s0->p.precision || s->plane != s0->plane ||
        ((s->t ^ s0->t) & 1) || s->stream != s0->stream)
      return vlb::set_error(VLB_EINVAL,
                            "vlb_batch_create: member %d differs in lattice, precision, coefficient mode, "
                            "time parity or stream",
                            i);
    if ((int64_t)m->md.q * m->ncell >= ((int64_t)1 << 31))
      return vlb::set_error(VLB_EINVAL, "vlb_batch_create: member %d is too large for a batch", i);
  }
  vlb_batch *b = new (std::nothrow) vlb_batch();
  if (!b) return vlb::set_error(VLB_ENOMEM, "vlb_batch_create: host allocation");
  b->sims.assign(sims, sims + nsims);
  b->stream = s0->stream;
  b->device = dev;
  std::vector<vlb::StepArgs> args;
  for (vlb_sim *s : b->sims) {
    args.push_back(s->mesh->md.q == 9 ? vlb::make_step_args<9>(s) : vlb::make_step_args<19>(s));
    b->cells += s->mesh->ncell;
  }
  cudaError_t e = cudaMalloc(&b->d_args, sizeof(vlb::StepArgs) * args.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_args, args.data(), sizeof(vlb::StepArgs) * args.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // default: about two runs per resident block
    const int64_t res = vlb::batch_resident(b);
    const int64_t tt = vlb::total_tiles(b);
    const int64_t run = (tt + 2 * res - 1) / (2 * res);
    e = vlb::set_run(b, run > 0 ? run : 1);
  }
  if (e != cudaSuccess) {
    vlb_batch_destroy(b);
    return vlb::set_error(e == cudaErrorMemoryAllocation ? VLB_ENOMEM : VLB_ECUDA, "vlb_batch_create: %s",
                          cudaGetErrorString(e));
  }
  *out = b;
  return VLB_OK;
}

int vlb_batch_step(vlb_batch *b, int64_t nsteps) {
  if (!b) return vlb::set_error(VLB_EINVAL, "vlb_batch_step: NULL batch");
  if (nsteps < 0) return vlb::set_error(VLB_EINVAL, "vlb_batch_step: nsteps < 0");
  const cudaError_t e = vlb::run_steps(b, nsteps);
  if (e != cudaSuccess) return vlb::set_error(VLB_ECUDA, "vlb_batch_step: %s", cudaGetErrorString(e));
  return VLB_OK;
}

int vlb_batch_tune(vlb_batch *b, int32_t steps, int64_t *run_length_out) {
  if (!b || steps < 1) return vlb::set_error(VLB_EINVAL, "vlb_batch_tune: NULL batch or steps < 1");
  const int64_t res = vlb::batch_resident(b);
  const int64_t tt = vlb::total_tiles(b);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.0f;
  int64_t best = b->run;
  // candidates: about 1, 2, 4 and 8 runs per resident block
  for (int k = 1; k <= 8 && e == cudaSuccess; k *= 2) {
    int64_t run = (tt + k * res - 1) / (k * res);
    if (run < 1) run = 1;
    e = vlb::set_run(b, run);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    const int64_t start = b->sims[0]->t;
    int64_t t = start;
    for (int32_t i = 0; i < steps && e == cudaSuccess; i++, t++) e = vlb::launch_one(b, (t & 1) != 0);
    for (vlb_sim *s : b->sims) s->t += t - start;
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (k == 1 || ms < best_ms)) {
      best_ms = ms;
      best = run;
    }
  }
  if (e == cudaSuccess) e = vlb::set_run(b, best);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return vlb::set_error(VLB_ECUDA, "vlb_batch_tune: %s", cudaGetErrorString(e));
  if (run_length_out) *run_length_out = b->run;
  return VLB_OK;
}

int vlb_batch_layout(const vlb_batch *b, int64_t *blocks, int64_t *run_length, int64_t *cells) {
  if (!b) return vlb::set_error(VLB_EINVAL, "vlb_batch_layout: NULL batch");
  if (blocks) *blocks = b->nitems;
  if (run_length) *run_length = b->run;
  if (cells) *cells = b->cells;
  return VLB_OK;
}

void vlb_batch_destroy(vlb_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_items) cudaFree(b->d_items);
  delete b;
}

}  // extern "C"

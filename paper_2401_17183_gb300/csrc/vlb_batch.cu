// vlb_batch.cu -- many simulations advanced by one kernel launch per time step.
//
// Each member's tiles are cut into runs of `run` tiles; every run is one block
// of a single launch of k_step_batch, which reads its member's kernel
// arguments from a device array. The block shape (tile width and the
// resident blocks the registers are cut for) and the run length are chosen
// by timing (vlb_batch_tune). The per-cell work is that of vlb_step, so a
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

// Block shapes the tuner chooses from: threads per block (the tile width,
// cells along the fastest axis) and the resident blocks per SM the register
// budget is cut for. Narrow tiles waste fewer threads at the ragged end of
// short rows; more resident blocks hide more latency if the code fits the
// smaller register budget. Shape 0 is the single-mesh step's.
struct BatchShape {
  int threads, min_blocks;
};
constexpr BatchShape kShapes32[] = {{128, 3}, {128, 6}, {128, 8}, {64, 12}};
constexpr BatchShape kShapes64[] = {{128, 2}, {64, 4}};
constexpr int kNShapes32 = sizeof(kShapes32) / sizeof(kShapes32[0]);
constexpr int kNShapes64 = sizeof(kShapes64) / sizeof(kShapes64[0]);

int nshapes(const BatchKind &k) { return k.f64 ? kNShapes64 : kNShapes32; }
BatchShape shape_of(const BatchKind &k, int i) { return k.f64 ? kShapes64[i] : kShapes32[i]; }

template <int Q, typename R, bool PLANE, int T, int MINB>
BatchKernel pick_t(bool odd) {
  return odd ? k_step_batch<Q, R, R, true, PLANE, int32_t, T, MINB>
             : k_step_batch<Q, R, R, false, PLANE, int32_t, T, MINB>;
}

template <int Q, typename R, bool PLANE>
BatchKernel pick_kernel(bool odd, int shape) {
  if constexpr (sizeof(R) == 8) {
    return shape == 1 ? pick_t<Q, R, PLANE, kShapes64[1].threads, kShapes64[1].min_blocks>(odd)
                      : pick_t<Q, R, PLANE, kShapes64[0].threads, kShapes64[0].min_blocks>(odd);
  } else {
    switch (shape) {
      case 1: return pick_t<Q, R, PLANE, kShapes32[1].threads, kShapes32[1].min_blocks>(odd);
      case 2: return pick_t<Q, R, PLANE, kShapes32[2].threads, kShapes32[2].min_blocks>(odd);
      case 3: return pick_t<Q, R, PLANE, kShapes32[3].threads, kShapes32[3].min_blocks>(odd);
      default: return pick_t<Q, R, PLANE, kShapes32[0].threads, kShapes32[0].min_blocks>(odd);
    }
  }
}

BatchKernel batch_kernel(const BatchKind &k, bool odd, int shape) {
  if (k.q == 9) {
    if (k.f64) return k.plane ? pick_kernel<9, double, true>(odd, shape) : pick_kernel<9, double, false>(odd, shape);
    return k.plane ? pick_kernel<9, float, true>(odd, shape) : pick_kernel<9, float, false>(odd, shape);
  }
  if (k.f64) return k.plane ? pick_kernel<19, double, true>(odd, shape) : pick_kernel<19, double, false>(odd, shape);
  return k.plane ? pick_kernel<19, float, true>(odd, shape) : pick_kernel<19, float, false>(odd, shape);
}

template <int Q, typename R>
size_t smem_q(int threads) {
  return threads == 64 ? sizeof(StepSmem<Q, R, R, 64>) : sizeof(StepSmem<Q, R, R, 128>);
}

size_t batch_smem(const BatchKind &k, int shape) {
  const int th = shape_of(k, shape).threads;
  if (k.q == 9) return k.f64 ? smem_q<9, double>(th) : smem_q<9, float>(th);
  return k.f64 ? smem_q<19, double>(th) : smem_q<19, float>(th);
}

BatchKind kind_of(const vlb_batch *b) {
  const vlb_sim *s = b->sims[0];
  return BatchKind{s->mesh->md.q, s->p.precision == VLB_F64, s->plane != 0};
}

int batch_threads(const vlb_batch *b) { return shape_of(kind_of(b), b->shape).threads; }

int64_t member_tiles(const vlb_sim *s, int threads) {
  const vlb_mesh *m = s->mesh;
  const int dim = m->md.dim;
  const int64_t nfast = m->md.n[dim - 1];
  const int64_t ntf = (nfast + threads - 1) / threads;
  return ntf * (dim == 3 ? m->md.n[0] * m->md.n[1] : m->md.n[0]);
}

int64_t total_tiles(const vlb_batch *b) {
  int64_t t = 0;
  const int th = batch_threads(b);
  for (const vlb_sim *s : b->sims) t += member_tiles(s, th);
  return t;
}

// blocks the batch kernel keeps resident on the device
int64_t batch_resident(const vlb_batch *b) {
  const BatchKind k = kind_of(b);
  return resident_blocks(reinterpret_cast<const void *>(batch_kernel(k, false, b->shape)),
                         batch_smem(k, b->shape), batch_threads(b));
}

// switch to block shape `shape`: the members' kernel arguments (their tile
// counts depend on the tile width) go to the device again
cudaError_t set_shape(vlb_batch *b, int shape) {
  b->shape = shape;
  const int th = batch_threads(b);
  std::vector<StepArgs> args;
  for (vlb_sim *s : b->sims)
    args.push_back(s->mesh->md.q == 9 ? make_step_args<9>(s, th) : make_step_args<19>(s, th));
  const size_t bytes = sizeof(StepArgs) * args.size();
  if (!b->d_args) {
    const cudaError_t e = cudaMalloc(&b->d_args, bytes);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_args, args.data(), bytes, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

// cut every member into runs of `run` tiles and upload the work list
cudaError_t set_run(vlb_batch *b, int64_t run) {
  std::vector<BatchItem> items;
  const int th = batch_threads(b);
  for (size_t m = 0; m < b->sims.size(); m++) {
    const int64_t nt = member_tiles(b->sims[m], th);
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

// default run length: about two runs per resident block
cudaError_t default_run(vlb_batch *b) {
  const int64_t res = batch_resident(b);
  const int64_t tt = total_tiles(b);
  const int64_t run = (tt + 2 * res - 1) / (2 * res);
  return set_run(b, run > 0 ? run : 1);
}

cudaError_t launch_one(const vlb_batch *b, bool odd) {
  const BatchKind k = kind_of(b);
  const BatchKernel kern = batch_kernel(k, odd, b->shape);
  kern<<<(unsigned)b->nitems, (unsigned)batch_threads(b), batch_smem(k, b->shape), b->stream>>>(
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
    p.func = reinterpret_cast<void *>(batch_kernel(k, (i & 1) != 0, b->shape));
    p.gridDim = dim3((unsigned)b->nitems);
    p.blockDim = dim3((unsigned)batch_threads(b));
    p.sharedMemBytes = (unsigned)batch_smem(k, b->shape);
    p.kernelParams = params;
    cudaGraphNode_t node;
    e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
    prev = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) {
    b->graph_run = b->run;
    b->graph_shape = b->shape;
  }
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
  if (e == cudaSuccess && n >= kGraphSteps && (!b->graph || b->graph_run != b->run || b->graph_shape != b->shape))
    e = build_graph(b);
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
  for (vlb_sim *s : b->sims) b->cells += s->mesh->ncell;
  cudaError_t e = vlb::set_shape(b, 0);
  if (e == cudaSuccess) e = vlb::default_run(b);
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
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.0f;
  int64_t best_run = b->run;
  int best_shape = b->shape;
  bool first = true;
  const int ns = vlb::nshapes(vlb::kind_of(b));
  // every block shape with run lengths of about 1, 2, 4 and 8 runs per
  // resident block
  for (int sh = 0; sh < ns && e == cudaSuccess; sh++) {
    e = vlb::set_shape(b, sh);
    const int64_t res = e == cudaSuccess ? vlb::batch_resident(b) : 1;
    const int64_t tt = vlb::total_tiles(b);
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
      if (e == cudaSuccess && (first || ms < best_ms)) {
        first = false;
        best_ms = ms;
        best_run = run;
        best_shape = sh;
      }
    }
  }
  if (e == cudaSuccess) e = vlb::set_shape(b, best_shape);
  if (e == cudaSuccess) e = vlb::set_run(b, best_run);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return vlb::set_error(VLB_ECUDA, "vlb_batch_tune: %s", cudaGetErrorString(e));
  if (run_length_out) *run_length_out = b->run;
  return VLB_OK;
}

int vlb_batch_tune_steps(const vlb_batch *b, int32_t steps, int64_t *advanced) {
  if (!b || steps < 1 || !advanced) return vlb::set_error(VLB_EINVAL, "vlb_batch_tune_steps: bad argument");
  *advanced = (int64_t)4 * vlb::nshapes(vlb::kind_of(b)) * steps;
  return VLB_OK;
}

int vlb_batch_set_shape(vlb_batch *b, int32_t shape) {
  if (!b) return vlb::set_error(VLB_EINVAL, "vlb_batch_set_shape: NULL batch");
  const int ns = vlb::nshapes(vlb::kind_of(b));
  if (shape < 0 || shape >= ns)
    return vlb::set_error(VLB_EINVAL, "vlb_batch_set_shape: shape %d outside [0, %d)", shape, ns);
  cudaError_t e = vlb::set_shape(b, shape);
  if (e == cudaSuccess) e = vlb::default_run(b);
  if (e != cudaSuccess) return vlb::set_error(VLB_ECUDA, "vlb_batch_set_shape: %s", cudaGetErrorString(e));
  return VLB_OK;
}

int vlb_batch_shape(const vlb_batch *b, int32_t *threads, int32_t *min_blocks) {
  if (!b) return vlb::set_error(VLB_EINVAL, "vlb_batch_shape: NULL batch");
  const vlb::BatchShape sh = vlb::shape_of(vlb::kind_of(b), b->shape);
  if (threads) *threads = sh.threads;
  if (min_blocks) *min_blocks = sh.min_blocks;
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

// vlb_nn.cu -- the learned warm start (include/vlb_nn.h): a 2D U-Net with
// hand-written forward and backward kernels. Weights and activations are
// stored in FP32 or bfloat16 and every product is accumulated in FP32; the
// optimizer (Adam) works on an FP32 master copy of the parameters.
//
// Kernels: a tiled direct convolution (3x3 or 1x1, zero padding) that also
// serves the backward pass with respect to its input (with transposed,
// flipped weights), a tiled weight-gradient reduction with fixed-order
// split sums (deterministic), 2x2 average pooling, 2x nearest upsampling,
// ReLU masks, bias gradients, the mean-square loss and Adam. Activations
// are NCHW with a batch stride, so a channel concatenation is a view into
// one buffer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/vlb.h"
#include "../../include/vlb_nn.h"

namespace vlb {
int set_error(int code, const char *fmt, ...);
}

namespace nn {

constexpr int kTile = 16;   // output pixels per block side
constexpr int kCo = 16;     // output channels per block
constexpr int kCi = 8;      // input channels per chunk
constexpr int kThreads = kTile * kTile;

template <typename T>
__device__ __forceinline__ float ld(const T *p) {
  return static_cast<float>(*p);
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
template <typename T>
__device__ __forceinline__ T st(float x) {
  return static_cast<T>(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 st<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// ---------------------------------------------------------------- convolution
// out[b][co][p] = act(bias[co] + sum_ci sum_k w[co][ci][k] in[b][ci][p + off_k])
// in: channel stride H*W, batch stride ibs; out likewise with obs.
// grid (tiles of W x H, ceil(Co / kCo), B), block kThreads.
template <int K, typename TI, typename TW, typename TO, bool RELU>
__global__ void __launch_bounds__(kThreads) k_conv(const TI *__restrict__ in, int64_t ibs, const TW *__restrict__ w,
                                                   const float *__restrict__ bias, TO *__restrict__ out, int64_t obs,
                                                   int Ci, int Co, int H, int W) {
  constexpr int R = K / 2, TS = kTile + 2 * R;
  __shared__ float in_s[kCi][TS][TS];
  __shared__ __align__(16) float w_s[kCi][K * K][kCo];
  const int tilesx = (W + kTile - 1) / kTile;
  const int tx0 = (blockIdx.x % tilesx) * kTile, ty0 = (blockIdx.x / tilesx) * kTile;
  const int co0 = blockIdx.y * kCo, b = blockIdx.z;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int64_t HW = (int64_t)H * W;
  const TI *inb = in + b * ibs;
  float acc[kCo];
#pragma unroll
  for (int o = 0; o < kCo; o++) acc[o] = 0.0f;
  for (int c0 = 0; c0 < Ci; c0 += kCi) {
    for (int i = threadIdx.x; i < kCi * TS * TS; i += kThreads) {
      const int c = i / (TS * TS), r = i % (TS * TS), yy = ty0 - R + r / TS, xx = tx0 - R + r % TS;
      float v = 0.0f;
      if (c0 + c < Ci && yy >= 0 && yy < H && xx >= 0 && xx < W) v = ld(inb + (c0 + c) * HW + (int64_t)yy * W + xx);
      in_s[c][r / TS][r % TS] = v;
    }
    for (int i = threadIdx.x; i < kCi * K * K * kCo; i += kThreads) {
      const int o = i % kCo, k = (i / kCo) % (K * K), c = i / (kCo * K * K);
      float v = 0.0f;
      if (c0 + c < Ci && co0 + o < Co) v = ld(w + ((int64_t)(co0 + o) * Ci + c0 + c) * K * K + k);
      w_s[c][k][o] = v;
    }
    __syncthreads();
#pragma unroll 2
    for (int c = 0; c < kCi; c++)
#pragma unroll
      for (int k = 0; k < K * K; k++) {
        const float v = in_s[c][ty + k / K][tx + k % K];
        const float4 *wv = reinterpret_cast<const float4 *>(&w_s[c][k][0]);
#pragma unroll
        for (int q = 0; q < kCo / 4; q++) {
          const float4 x = wv[q];
          acc[4 * q] = fmaf(v, x.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(v, x.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(v, x.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(v, x.w, acc[4 * q + 3]);
        }
      }
    __syncthreads();
  }
  const int y = ty0 + ty, x = tx0 + tx;
  if (y >= H || x >= W) return;
  TO *ob = out + b * obs + (int64_t)y * W + x;
#pragma unroll
  for (int o = 0; o < kCo; o++) {
    if (co0 + o >= Co) break;
    float v = acc[o] + (bias ? bias[co0 + o] : 0.0f);
    if (RELU) v = fmaxf(v, 0.0f);
    ob[(int64_t)(co0 + o) * HW] = st<TO>(v);
  }
}

// ------------------------------------------------- tensor-core convolution
// The 3x3 forward convolution of bfloat16 activations and weights as an
// implicit GEMM on the fifth-generation tensor cores (tcgen05, sm_100 and
// later): for the 128 output pixels p of a tile and kk = ci * 9 + tap,
//   D[p][co] = sum_kk A[p][kk] B[co][kk],  A = the input patches (gathered
//   on the fly), B = w[co][ci][tap] (K-contiguous as stored),
// one MMA of M = 128, N = Co, K = 16 per step, FP32 accumulators in tensor
// memory. The operands go through two shared-memory stages in the
// no-swizzle K-major layout of 8-row x 16-byte core matrices (core (r/8,
// k/8) at (r/8) * 256 + (k/8) * 128 bytes), each stage guarded by an mbarrier
// that the MMA's commit arrives on. Every wait is bounded in time; a block
// that gives up sets *err, waits (bounded) for its own MMAs and frees its
// tensor memory.
constexpr int kTcM = 128;   // output pixels per tile (MMA M)
constexpr uint64_t kTcWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// shared-memory matrix descriptor: start address, leading (K-direction)
// byte offset 128 and stride (M/N-direction) byte offset 256, all >> 4; the
// descriptor version bit (46); no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ int core_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// wait until the mbarrier has completed the phase of the given parity, at
// most until t0 + kTcWaitNs; returns whether it did
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t t0) {
  uint32_t done = 0;
  while (true) {
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
    if (gtimer() - t0 > kTcWaitNs) return false;
  }
}
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// out[b][co][p] = act(bias[co] + sum_ci sum_tap w[co][ci][tap] in[b][ci][p + off_tap])
// for Co = N output channels; grid (H * W / 128, B), block 128 (thread t
// gathers the patch of pixel p0 + t and, in the epilogue, reads TMEM lane t).
// Needs H * W a multiple of 128, Ci a multiple of 8 (16-byte weight pieces)
// and 16-byte aligned weights.
template <int N, bool RELU>
__global__ void __launch_bounds__(kTcM) k_conv3_tc(const __nv_bfloat16 *__restrict__ in, int64_t ibs,
                                                  const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
                                                  __nv_bfloat16 *__restrict__ out, int64_t obs, int Ci, int H, int W,
                                                  int *err) {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "MMA N for M = 128");
  constexpr int TCOLS = N < 32 ? 32 : N;   // tensor-memory columns: a power of two, at least 32
  static_assert((TCOLS & (TCOLS - 1)) == 0, "N must be a power of two");
  __shared__ __align__(1024) unsigned char sA[2][kTcM * 32];
  __shared__ __align__(1024) unsigned char sB[2][N * 32];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int HW = H * W, p = blockIdx.x * kTcM + tid, b = blockIdx.y;
  const int y = p / W, x = p - y * W;
  const int K9 = Ci * 9, nch = (K9 + 15) / 16;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  // instruction descriptor: FP32 accumulators, bfloat16 A and B, both
  // K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const __nv_bfloat16 *inb = in + (int64_t)b * ibs;
  // the operands of step j in registers: this pixel's 16 patch values as
  // bfloat16 pairs, and this thread's 16-byte weight pieces; they are loaded
  // one step ahead, so that their latency overlaps the previous MMA
  constexpr int NQ = (2 * N + kTcM - 1) / kTcM;   // weight pieces per thread
  uint32_t pa[8];
  uint4 pb[NQ];
  auto load_step = [&](int j) {
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
      __nv_bfloat16 v2[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int kk = j * 16 + e + u;
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (kk < K9) {
          const int ci = kk / 9, tap = kk - ci * 9;
          const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
          if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = inb[(int64_t)ci * HW + yy * W + xx];
        }
        v2[u] = v;
      }
      pa[e / 2] = pack_bf16(v2[0], v2[1]);
    }
    // (a piece lies wholly inside or wholly past the row end: 9 Ci is a
    // multiple of 8)
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      const int q = tid + i * kTcM, kk0 = j * 16 + (q & 1) * 8;
      pb[i] = make_uint4(0u, 0u, 0u, 0u);
      if (q < 2 * N && kk0 < K9) pb[i] = *reinterpret_cast<const uint4 *>(w + (int64_t)(q >> 1) * K9 + kk0);
    }
  };
  const uint64_t t0 = gtimer();
  bool ok = true;
  int issued = 0;
  load_step(0);
  for (int j = 0; j < nch; j++) {
    const int s = j & 1;
    // the MMA of step j - 2 read this stage
    bool late = false;
    if (j >= 2) late = !mbar_wait(smem_u32(&bar[s]), ((j - 2) >> 1) & 1, t0);
    if (__syncthreads_or(late)) {
      ok = false;
      break;
    }
    // A: two 16-byte pieces of this pixel's row; B: this thread's weight pieces
    *reinterpret_cast<uint4 *>(&sA[s][core_off(tid, 0)]) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
    *reinterpret_cast<uint4 *>(&sA[s][core_off(tid, 8)]) = make_uint4(pa[4], pa[5], pa[6], pa[7]);
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      const int q = tid + i * kTcM;
      if (q < 2 * N) *reinterpret_cast<uint4 *>(&sB[s][core_off(q >> 1, (q & 1) * 8)]) = pb[i];
    }
    // the stores above are read by the tensor cores (the async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(umma_desc(smem_u32(&sA[s][0]))), "l"(umma_desc(smem_u32(&sB[s][0]))), "r"(idesc), "r"(j > 0 ? 1 : 0));
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar[s]))
                   : "memory");
    }
    issued = j + 1;
    if (j + 1 < nch) load_step(j + 1);
  }
  // the last MMA done (its commit also covers every earlier one)
  bool late = false;
  if (issued > 0) late = !mbar_wait(smem_u32(&bar[(issued - 1) & 1]), ((issued - 1) >> 1) & 1, gtimer());
  if (__syncthreads_or(late)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && issued == nch) {
    // epilogue: warp w reads TMEM lanes 32w.. (pixels), 16 channels at a time
    __nv_bfloat16 *ob = out + (int64_t)b * obs + p;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 16; u++) {
        float v = __uint_as_float(r[u]) + (bias ? bias[c0 + u] : 0.0f);
        if (RELU) v = fmaxf(v, 0.0f);
        ob[(int64_t)(c0 + u) * HW] = __float2bfloat16_rn(v);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// wt[ci][co][k'] = w[co][ci][K*K - 1 - k'] (FP32): the weights of the
// backward pass with respect to the input
template <typename TW>
__global__ void k_transpose_flip(const TW *__restrict__ w, float *__restrict__ wt, int Ci, int Co, int KK) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Ci * Co * KK) return;
  const int k = (int)(i % KK), co = (int)((i / KK) % Co), ci = (int)(i / ((int64_t)KK * Co));
  wt[i] = ld(w + ((int64_t)co * Ci + ci) * KK + (KK - 1 - k));
}

// Weight gradient partials: dwp[split][co][ci][k] = sum over this split's
// (sample, pixel tile) pairs of g[b][co][p] in[b][ci][p + off_k].
// grid (ceil(Co/16), ceil(Ci/8), nsplit), block 128: thread (co, ci).
template <int K, typename TI>
__global__ void __launch_bounds__(128) k_conv_dw(const TI *__restrict__ in, int64_t ibs, const float *__restrict__ g,
                                                 int64_t gbs, float *__restrict__ dwp, int Ci, int Co, int H, int W,
                                                 int B) {
  constexpr int R = K / 2, TS = kTile + 2 * R;
  __shared__ float g_s[16][kTile * kTile + 1];
  __shared__ float in_s[8][TS * TS + 1];
  const int co0 = blockIdx.x * 16, ci0 = blockIdx.y * 8;
  const int tco = threadIdx.x / 8, tci = threadIdx.x % 8;
  const int tilesx = (W + kTile - 1) / kTile, tilesy = (H + kTile - 1) / kTile;
  const int64_t HW = (int64_t)H * W;
  const int64_t nwork = (int64_t)B * tilesx * tilesy;
  float acc[K * K];
#pragma unroll
  for (int k = 0; k < K * K; k++) acc[k] = 0.0f;
  for (int64_t wk = blockIdx.z; wk < nwork; wk += gridDim.z) {
    const int b = (int)(wk / (tilesx * tilesy)), tl = (int)(wk % (tilesx * tilesy));
    const int tx0 = (tl % tilesx) * kTile, ty0 = (tl / tilesx) * kTile;
    for (int i = threadIdx.x; i < 16 * kTile * kTile; i += 128) {
      const int o = i / (kTile * kTile), p = i % (kTile * kTile), yy = ty0 + p / kTile, xx = tx0 + p % kTile;
      float v = 0.0f;
      if (co0 + o < Co && yy < H && xx < W) v = g[b * gbs + (co0 + o) * HW + (int64_t)yy * W + xx];
      g_s[o][p] = v;
    }
    for (int i = threadIdx.x; i < 8 * TS * TS; i += 128) {
      const int c = i / (TS * TS), r = i % (TS * TS), yy = ty0 - R + r / TS, xx = tx0 - R + r % TS;
      float v = 0.0f;
      if (ci0 + c < Ci && yy >= 0 && yy < H && xx >= 0 && xx < W) v = ld(in + b * ibs + (ci0 + c) * HW + (int64_t)yy * W + xx);
      in_s[c][r] = v;
    }
    __syncthreads();
    for (int p = 0; p < kTile * kTile; p++) {
      const float gv = g_s[tco][p];
      const int py = p / kTile, px = p % kTile;
#pragma unroll
      for (int k = 0; k < K * K; k++) acc[k] = fmaf(gv, in_s[tci][(py + k / K) * TS + px + k % K], acc[k]);
    }
    __syncthreads();
  }
  if (co0 + tco < Co && ci0 + tci < Ci) {
    float *o = dwp + (((int64_t)blockIdx.z * Co + co0 + tco) * Ci + ci0 + tci) * (K * K);
#pragma unroll
    for (int k = 0; k < K * K; k++) o[k] = acc[k];
  }
}

// dst[i] = sum_s src[s][i] in split order (deterministic)
__global__ void k_sum_splits(const float *__restrict__ src, int nsplit, int64_t n, float *__restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int k = 0; k < nsplit; k++) s += src[k * n + i];
  dst[i] = s;
}

// db[co] = sum_b sum_p g[b][co][p]; one block per channel, fixed-order tree
__global__ void k_bias_grad(const float *__restrict__ g, int64_t gbs, int64_t HW, int B, float *__restrict__ db) {
  __shared__ float sh[256];
  const int co = blockIdx.x;
  float s = 0.0f;
  for (int b = 0; b < B; b++)
    for (int64_t p = threadIdx.x; p < HW; p += 256) s += g[b * gbs + co * HW + p];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[co] = sh[0];
}

// g *= (act > 0) over C channels of B samples
template <typename TA>
__global__ void k_relu_mask(float *__restrict__ g, int64_t gbs, const TA *__restrict__ act, int64_t abs_, int64_t CHW,
                            int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= CHW * B) return;
  const int64_t b = i / CHW, r = i % CHW;
  if (!(ld(act + b * abs_ + r) > 0.0f)) g[b * gbs + r] = 0.0f;
}

// 2x2 average pool: out [C][H/2][W/2] from in [C][H][W]
template <typename T>
__global__ void k_pool(const T *__restrict__ in, int64_t ibs, T *__restrict__ out, int64_t obs, int C, int H, int W,
                       int B) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t n = (int64_t)B * C * Ho * Wo;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % Wo), y = (int)((i / Wo) % Ho), c = (int)((i / ((int64_t)Wo * Ho)) % C);
  const int64_t b = i / ((int64_t)Wo * Ho * C);
  const T *p = in + b * ibs + (int64_t)c * H * W + (int64_t)(2 * y) * W + 2 * x;
  const float v = 0.25f * (ld(p) + ld(p + 1) + ld(p + W) + ld(p + W + 1));
  out[b * obs + (int64_t)c * Ho * Wo + (int64_t)y * Wo + x] = st<T>(v);
}

// gradient of the pool: gin[..] += gout / 4 (gin FP32)
__global__ void k_pool_bwd(const float *__restrict__ gout, int64_t gobs, float *__restrict__ gin, int64_t gibs, int C,
                           int H, int W, int B) {
  const int64_t n = (int64_t)B * C * H * W;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % W), y = (int)((i / W) % H), c = (int)((i / ((int64_t)W * H)) % C);
  const int64_t b = i / ((int64_t)W * H * C);
  gin[b * gibs + (int64_t)c * H * W + (int64_t)y * W + x] +=
      0.25f * gout[b * gobs + (int64_t)c * (H / 2) * (W / 2) + (int64_t)(y / 2) * (W / 2) + x / 2];
}

// 2x nearest upsampling: out [C][2h][2w] from in [C][h][w]
template <typename T>
__global__ void k_up(const T *__restrict__ in, int64_t ibs, T *__restrict__ out, int64_t obs, int C, int h, int w,
                     int B) {
  const int64_t n = (int64_t)B * C * 4 * h * w;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int W2 = 2 * w, H2 = 2 * h;
  const int x = (int)(i % W2), y = (int)((i / W2) % H2), c = (int)((i / ((int64_t)W2 * H2)) % C);
  const int64_t b = i / ((int64_t)W2 * H2 * C);
  out[b * obs + (int64_t)c * H2 * W2 + (int64_t)y * W2 + x] = in[b * ibs + (int64_t)c * h * w + (int64_t)(y / 2) * w + x / 2];
}

// gradient of the upsampling: gin[c][y][x] = sum of the four children (assigns)
__global__ void k_up_bwd(const float *__restrict__ gout, int64_t gobs, float *__restrict__ gin, int64_t gibs, int C,
                         int h, int w, int B) {
  const int64_t n = (int64_t)B * C * h * w;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % w), y = (int)((i / w) % h), c = (int)((i / ((int64_t)w * h)) % C);
  const int64_t b = i / ((int64_t)w * h * C);
  const float *p = gout + b * gobs + (int64_t)c * 4 * h * w + (int64_t)(2 * y) * (2 * w) + 2 * x;
  gin[b * gibs + (int64_t)c * h * w + (int64_t)y * w + x] = p[0] + p[1] + p[2 * w] + p[2 * w + 1];
}

template <typename TO>
__global__ void k_convert(const float *__restrict__ in, TO *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = st<TO>(in[i]);
}

// dst[b][r] = src[b][r] (converted) for r < CHW: the input into its view
template <typename TO>
__global__ void k_convert_into(const float *__restrict__ src, int64_t sbs, TO *__restrict__ dst, int64_t dbs,
                               int64_t CHW, int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= CHW * B) return;
  const int64_t b = i / CHW, r = i % CHW;
  dst[b * dbs + r] = st<TO>(src[b * sbs + r]);
}

// dst[b][r] += src[b][r] for a channel block (between views)
__global__ void k_add_into(const float *__restrict__ src, int64_t sbs, float *__restrict__ dst, int64_t dbs, int64_t CHW,
                           int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= CHW * B) return;
  const int64_t b = i / CHW, r = i % CHW;
  dst[b * dbs + r] += src[b * sbs + r];
}

// mean-square loss: partial sums per block and dy = 2 (y - t) / n
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy, int64_t n,
                      double *__restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d / (float)n;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// He-uniform initial weights from SplitMix64 (counter = parameter index)
__global__ void k_init_params(float *p, int64_t off, int64_t n, float bound, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(off + i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  p[off + i] = (float)((2.0 * u - 1.0) * bound);
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace nn

// ------------------------------------------------------------------ host side
struct NNLayer {
  int cin, cout, k, h, w;  // input channels, output channels, kernel, grid at this layer
  int64_t woff, boff;       // offsets in the parameter vector
};

// an activation buffer (storage T) or gradient buffer (FP32) view
struct View {
  int64_t off;    // element offset of channel 0 in its buffer
  int64_t bs;     // batch stride (elements)
};

struct vlb_nn {
  int ci, co, width, H, W, maxb, storage;
  std::vector<NNLayer> L;
  int64_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master params, grads, Adam moments
  void *pc = nullptr;        // compute copy of the parameters (bfloat16) or NULL
  void *act = nullptr;       // activations (storage type)
  float *gr = nullptr;       // gradients of activations (FP32)
  float *wt = nullptr;       // transposed weights (FP32), largest layer
  float *dwp = nullptr;      // weight-gradient split partials
  double *lossp = nullptr;
  int64_t act_n = 0, wt_n = 0, dwp_n = 0;
  int nsplit = 16;
  int *d_err = nullptr;      // set by a tensor-core convolution that gave up waiting
  int tc = 1;                // 3x3 forward convolutions in bfloat16 on the tensor cores where they fit
  // activation views (offsets in act / gr), per sample sizes
  View x_in, e1, c1, s1, p1, e2, c2, s2, p2, e3, b3, d2, t2, d1, t1;
};

namespace {

#define NN_CU(x)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess)                                                                        \
      return vlb::set_error(e_ == cudaErrorMemoryAllocation ? VLB_ENOMEM : VLB_ECUDA, "%s: %s", #x, \
                            cudaGetErrorString(e_));                                              \
  } while (0)

// the tensor-core form of a 3x3 layer (bfloat16 storage): Co a power of two
// in [16, 256], H * W a multiple of 128, Ci a multiple of 8 and the layer's
// weights 16-byte aligned
inline bool tc_fits(const vlb_nn *n, const NNLayer &l) {
  const bool pow2 = l.cout >= 16 && l.cout <= 256 && (l.cout & (l.cout - 1)) == 0;
  // (16-byte weight pieces: the layer's weights start on a multiple of 8 elements)
  return n->tc && n->storage == VLB_NN_BF16 && l.k == 3 && pow2 && ((int64_t)l.h * l.w) % nn::kTcM == 0 &&
         l.cin % 8 == 0 && l.woff % 8 == 0;
}

template <int N>
void launch_tc(const vlb_nn *n, const NNLayer &l, const __nv_bfloat16 *in, int64_t ibs, const __nv_bfloat16 *w,
               const float *bias, __nv_bfloat16 *out, int64_t obs, bool relu, int B) {
  const dim3 grid((unsigned)((int64_t)l.h * l.w / nn::kTcM), (unsigned)B);
  if (relu)
    nn::k_conv3_tc<N, true><<<grid, nn::kTcM>>>(in, ibs, w, bias, out, obs, l.cin, l.h, l.w, n->d_err);
  else
    nn::k_conv3_tc<N, false><<<grid, nn::kTcM>>>(in, ibs, w, bias, out, obs, l.cin, l.h, l.w, n->d_err);
}

template <typename T>
int conv(const vlb_nn *n, const NNLayer &l, const T *in, int64_t ibs, const void *w, const float *bias, void *out,
         int64_t obs, bool relu, bool out_f32, int B) {
  if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    if (tc_fits(n, l)) {
      const __nv_bfloat16 *wb = static_cast<const __nv_bfloat16 *>(w);
      __nv_bfloat16 *ob = static_cast<__nv_bfloat16 *>(out);
      switch (l.cout) {
        case 16: launch_tc<16>(n, l, in, ibs, wb, bias, ob, obs, relu, B); break;
        case 32: launch_tc<32>(n, l, in, ibs, wb, bias, ob, obs, relu, B); break;
        case 64: launch_tc<64>(n, l, in, ibs, wb, bias, ob, obs, relu, B); break;
        case 128: launch_tc<128>(n, l, in, ibs, wb, bias, ob, obs, relu, B); break;
        default: launch_tc<256>(n, l, in, ibs, wb, bias, ob, obs, relu, B); break;
      }
      NN_CU(cudaGetLastError());
      return VLB_OK;
    }
  }
  const dim3 grid((unsigned)(((l.w + nn::kTile - 1) / nn::kTile) * ((l.h + nn::kTile - 1) / nn::kTile)),
                  (unsigned)((l.cout + nn::kCo - 1) / nn::kCo), (unsigned)B);
  const bool bf = n->storage == VLB_NN_BF16;
  if (l.k == 3) {
    if (bf) {
      if (relu)
        nn::k_conv<3, T, __nv_bfloat16, T, true><<<grid, nn::kThreads>>>(
            in, ibs, (const __nv_bfloat16 *)w, bias, (T *)out, obs, l.cin, l.cout, l.h, l.w);
      else
        nn::k_conv<3, T, __nv_bfloat16, T, false><<<grid, nn::kThreads>>>(
            in, ibs, (const __nv_bfloat16 *)w, bias, (T *)out, obs, l.cin, l.cout, l.h, l.w);
    } else {
      if (relu)
        nn::k_conv<3, T, float, T, true><<<grid, nn::kThreads>>>(in, ibs, (const float *)w, bias, (T *)out, obs, l.cin,
                                                                  l.cout, l.h, l.w);
      else
        nn::k_conv<3, T, float, T, false><<<grid, nn::kThreads>>>(in, ibs, (const float *)w, bias, (T *)out, obs,
                                                                   l.cin, l.cout, l.h, l.w);
    }
  } else {
    // the 1x1 head writes FP32 outputs
    if (bf)
      nn::k_conv<1, T, __nv_bfloat16, float, false><<<grid, nn::kThreads>>>(
          in, ibs, (const __nv_bfloat16 *)w, bias, (float *)out, obs, l.cin, l.cout, l.h, l.w);
    else
      nn::k_conv<1, T, float, float, false><<<grid, nn::kThreads>>>(in, ibs, (const float *)w, bias, (float *)out,
                                                                   obs, l.cin, l.cout, l.h, l.w);
  }
  (void)out_f32;
  NN_CU(cudaGetLastError());
  return VLB_OK;
}

// gradient with respect to the input of layer l: gin = conv(gout; w^T flipped)
int conv_bwd_data(vlb_nn *n, const NNLayer &l, const float *gout, int64_t gobs, float *gin, int64_t gibs, int B) {
  const int KK = l.k * l.k;
  const int64_t nw = (int64_t)l.cin * l.cout * KK;
  if (n->storage == VLB_NN_BF16)
    nn::k_transpose_flip<__nv_bfloat16><<<nn::nblk(nw), 256>>>((const __nv_bfloat16 *)n->pc + l.woff, n->wt, l.cin,
                                                                l.cout, KK);
  else
    nn::k_transpose_flip<float><<<nn::nblk(nw), 256>>>(n->p + l.woff, n->wt, l.cin, l.cout, KK);
  NN_CU(cudaGetLastError());
  const dim3 grid((unsigned)(((l.w + nn::kTile - 1) / nn::kTile) * ((l.h + nn::kTile - 1) / nn::kTile)),
                  (unsigned)((l.cin + nn::kCo - 1) / nn::kCo), (unsigned)B);
  if (l.k == 3)
    nn::k_conv<3, float, float, float, false><<<grid, nn::kThreads>>>(gout, gobs, n->wt, nullptr, gin, gibs, l.cout,
                                                                      l.cin, l.h, l.w);
  else
    nn::k_conv<1, float, float, float, false><<<grid, nn::kThreads>>>(gout, gobs, n->wt, nullptr, gin, gibs, l.cout,
                                                                      l.cin, l.h, l.w);
  NN_CU(cudaGetLastError());
  return VLB_OK;
}

// weight and bias gradients of layer l from its input (activations) and gout
template <typename T>
int conv_bwd_weight(vlb_nn *n, const NNLayer &l, const T *in, int64_t ibs, const float *gout, int64_t gobs, int B) {
  const int KK = l.k * l.k;
  const dim3 grid((unsigned)((l.cout + 15) / 16), (unsigned)((l.cin + 7) / 8), (unsigned)n->nsplit);
  if (l.k == 3)
    nn::k_conv_dw<3, T><<<grid, 128>>>(in, ibs, gout, gobs, n->dwp, l.cin, l.cout, l.h, l.w, B);
  else
    nn::k_conv_dw<1, T><<<grid, 128>>>(in, ibs, gout, gobs, n->dwp, l.cin, l.cout, l.h, l.w, B);
  NN_CU(cudaGetLastError());
  const int64_t nw = (int64_t)l.cout * l.cin * KK;
  nn::k_sum_splits<<<nn::nblk(nw), 256>>>(n->dwp, n->nsplit, nw, n->g + l.woff);
  NN_CU(cudaGetLastError());
  nn::k_bias_grad<<<l.cout, 256>>>(gout, gobs, (int64_t)l.h * l.w, B, n->g + l.boff);
  NN_CU(cudaGetLastError());
  return VLB_OK;
}

template <typename T>
int relu_mask(float *g, int64_t gbs, const T *act, int64_t abs_, int C, int H, int W, int B) {
  const int64_t chw = (int64_t)C * H * W;
  nn::k_relu_mask<T><<<nn::nblk(chw * B), 256>>>(g, gbs, act, abs_, chw, B);
  NN_CU(cudaGetLastError());
  return VLB_OK;
}

#define NN_TRY(x)          \
  do {                     \
    const int rc_ = (x);   \
    if (rc_) return rc_;   \
  } while (0)

template <typename T>
int forward_t(vlb_nn *n, const float *d_x, float *d_y, int B) {
  T *A = static_cast<T *>(n->act);
  const void *Wp = n->storage == VLB_NN_BF16 ? n->pc : (const void *)n->p;
  auto wp = [&](const NNLayer &l) -> const void * {
    return n->storage == VLB_NN_BF16 ? (const void *)((const __nv_bfloat16 *)Wp + l.woff)
                                     : (const void *)((const float *)Wp + l.woff);
  };
  const int w = n->width, H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
  const auto &L = n->L;
  // input in the storage type
  const int64_t chw = (int64_t)n->ci * H * W;
  nn::k_convert_into<T><<<nn::nblk(chw * B), 256>>>(d_x, chw, A + n->x_in.off, n->x_in.bs, chw, B);
  NN_CU(cudaGetLastError());
  NN_TRY(conv<T>(n, L[0], A + n->x_in.off, n->x_in.bs, wp(L[0]), n->p + L[0].boff, A + n->e1.off, n->e1.bs, true, false, B));
  NN_TRY(conv<T>(n, L[1], A + n->e1.off, n->e1.bs, wp(L[1]), n->p + L[1].boff, A + n->s1.off, n->s1.bs, true, false, B));
  nn::k_pool<T><<<nn::nblk((int64_t)B * w * H2 * W2), 256>>>(A + n->s1.off, n->s1.bs, A + n->p1.off, n->p1.bs, w, H, W, B);
  NN_CU(cudaGetLastError());
  NN_TRY(conv<T>(n, L[2], A + n->p1.off, n->p1.bs, wp(L[2]), n->p + L[2].boff, A + n->e2.off, n->e2.bs, true, false, B));
  NN_TRY(conv<T>(n, L[3], A + n->e2.off, n->e2.bs, wp(L[3]), n->p + L[3].boff, A + n->s2.off, n->s2.bs, true, false, B));
  nn::k_pool<T><<<nn::nblk((int64_t)B * 2 * w * H4 * W4), 256>>>(A + n->s2.off, n->s2.bs, A + n->p2.off, n->p2.bs, 2 * w,
                                                                  H2, W2, B);
  NN_CU(cudaGetLastError());
  NN_TRY(conv<T>(n, L[4], A + n->p2.off, n->p2.bs, wp(L[4]), n->p + L[4].boff, A + n->e3.off, n->e3.bs, true, false, B));
  NN_TRY(conv<T>(n, L[5], A + n->e3.off, n->e3.bs, wp(L[5]), n->p + L[5].boff, A + n->b3.off, n->b3.bs, true, false, B));
  // c2 = [up(b3), s2]: s2 already sits in its slice
  nn::k_up<T><<<nn::nblk((int64_t)B * 4 * w * H2 * W2), 256>>>(A + n->b3.off, n->b3.bs, A + n->c2.off, n->c2.bs, 4 * w,
                                                                H4, W4, B);
  NN_CU(cudaGetLastError());
  NN_TRY(conv<T>(n, L[6], A + n->c2.off, n->c2.bs, wp(L[6]), n->p + L[6].boff, A + n->d2.off, n->d2.bs, true, false, B));
  NN_TRY(conv<T>(n, L[7], A + n->d2.off, n->d2.bs, wp(L[7]), n->p + L[7].boff, A + n->t2.off, n->t2.bs, true, false, B));
  nn::k_up<T><<<nn::nblk((int64_t)B * 2 * w * H * W), 256>>>(A + n->t2.off, n->t2.bs, A + n->c1.off, n->c1.bs, 2 * w, H2,
                                                              W2, B);
  NN_CU(cudaGetLastError());
  NN_TRY(conv<T>(n, L[8], A + n->c1.off, n->c1.bs, wp(L[8]), n->p + L[8].boff, A + n->d1.off, n->d1.bs, true, false, B));
  NN_TRY(conv<T>(n, L[9], A + n->d1.off, n->d1.bs, wp(L[9]), n->p + L[9].boff, A + n->t1.off, n->t1.bs, true, false, B));
  NN_TRY(conv<T>(n, L[10], A + n->t1.off, n->t1.bs, wp(L[10]), n->p + L[10].boff, d_y, (int64_t)n->co * H * W, false,
                 true, B));
  NN_CU(cudaDeviceSynchronize());
  int err = 0;
  NN_CU(cudaMemcpy(&err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    cudaMemset(n->d_err, 0, sizeof(int));
    return vlb::set_error(VLB_ECUDA, "vlb_nn_forward: a tensor-core convolution gave up waiting for its MMAs");
  }
  return VLB_OK;
}

template <typename T>
int backward_t(vlb_nn *n, const float *d_dy, int B) {
  const T *A = static_cast<const T *>(n->act);
  float *G = n->gr;
  const int w = n->width, H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
  const auto &L = n->L;
  const int64_t ybs = (int64_t)n->co * H * W;
  NN_CU(cudaMemset(G, 0, sizeof(float) * n->act_n));
  // head
  NN_TRY(conv_bwd_weight<T>(n, L[10], A + n->t1.off, n->t1.bs, d_dy, ybs, B));
  NN_TRY(conv_bwd_data(n, L[10], d_dy, ybs, G + n->t1.off, n->t1.bs, B));
  // t1 = relu(conv(d1))
  NN_TRY(relu_mask<T>(G + n->t1.off, n->t1.bs, A + n->t1.off, n->t1.bs, w, H, W, B));
  NN_TRY(conv_bwd_weight<T>(n, L[9], A + n->d1.off, n->d1.bs, G + n->t1.off, n->t1.bs, B));
  NN_TRY(conv_bwd_data(n, L[9], G + n->t1.off, n->t1.bs, G + n->d1.off, n->d1.bs, B));
  // d1 = relu(conv(c1))
  NN_TRY(relu_mask<T>(G + n->d1.off, n->d1.bs, A + n->d1.off, n->d1.bs, w, H, W, B));
  NN_TRY(conv_bwd_weight<T>(n, L[8], A + n->c1.off, n->c1.bs, G + n->d1.off, n->d1.bs, B));
  NN_TRY(conv_bwd_data(n, L[8], G + n->d1.off, n->d1.bs, G + n->c1.off, n->c1.bs, B));
  // c1 = [up(t2), s1]: gradient of t2 from the first 2w channels; s1's part stays in its slice
  nn::k_up_bwd<<<nn::nblk((int64_t)B * 2 * w * H2 * W2), 256>>>(G + n->c1.off, n->c1.bs, G + n->t2.off, n->t2.bs, 2 * w,
                                                                 H2, W2, B);
  NN_CU(cudaGetLastError());
  // t2 = relu(conv(d2))
  NN_TRY(relu_mask<T>(G + n->t2.off, n->t2.bs, A + n->t2.off, n->t2.bs, 2 * w, H2, W2, B));
  NN_TRY(conv_bwd_weight<T>(n, L[7], A + n->d2.off, n->d2.bs, G + n->t2.off, n->t2.bs, B));
  NN_TRY(conv_bwd_data(n, L[7], G + n->t2.off, n->t2.bs, G + n->d2.off, n->d2.bs, B));
  // d2 = relu(conv(c2))
  NN_TRY(relu_mask<T>(G + n->d2.off, n->d2.bs, A + n->d2.off, n->d2.bs, 2 * w, H2, W2, B));
  NN_TRY(conv_bwd_weight<T>(n, L[6], A + n->c2.off, n->c2.bs, G + n->d2.off, n->d2.bs, B));
  NN_TRY(conv_bwd_data(n, L[6], G + n->d2.off, n->d2.bs, G + n->c2.off, n->c2.bs, B));
  // c2 = [up(b3), s2]
  nn::k_up_bwd<<<nn::nblk((int64_t)B * 4 * w * H4 * W4), 256>>>(G + n->c2.off, n->c2.bs, G + n->b3.off, n->b3.bs, 4 * w,
                                                                 H4, W4, B);
  NN_CU(cudaGetLastError());
  // b3 = relu(conv(e3))
  NN_TRY(relu_mask<T>(G + n->b3.off, n->b3.bs, A + n->b3.off, n->b3.bs, 4 * w, H4, W4, B));
  NN_TRY(conv_bwd_weight<T>(n, L[5], A + n->e3.off, n->e3.bs, G + n->b3.off, n->b3.bs, B));
  NN_TRY(conv_bwd_data(n, L[5], G + n->b3.off, n->b3.bs, G + n->e3.off, n->e3.bs, B));
  // e3 = relu(conv(p2))
  NN_TRY(relu_mask<T>(G + n->e3.off, n->e3.bs, A + n->e3.off, n->e3.bs, 4 * w, H4, W4, B));
  NN_TRY(conv_bwd_weight<T>(n, L[4], A + n->p2.off, n->p2.bs, G + n->e3.off, n->e3.bs, B));
  NN_TRY(conv_bwd_data(n, L[4], G + n->e3.off, n->e3.bs, G + n->p2.off, n->p2.bs, B));
  // p2 = pool(s2): add into s2's gradient (its slice of c2)
  nn::k_pool_bwd<<<nn::nblk((int64_t)B * 2 * w * H2 * W2), 256>>>(G + n->p2.off, n->p2.bs, G + n->s2.off, n->s2.bs,
                                                                   2 * w, H2, W2, B);
  NN_CU(cudaGetLastError());
  // s2 = relu(conv(e2))
  NN_TRY(relu_mask<T>(G + n->s2.off, n->s2.bs, A + n->s2.off, n->s2.bs, 2 * w, H2, W2, B));
  NN_TRY(conv_bwd_weight<T>(n, L[3], A + n->e2.off, n->e2.bs, G + n->s2.off, n->s2.bs, B));
  NN_TRY(conv_bwd_data(n, L[3], G + n->s2.off, n->s2.bs, G + n->e2.off, n->e2.bs, B));
  // e2 = relu(conv(p1))
  NN_TRY(relu_mask<T>(G + n->e2.off, n->e2.bs, A + n->e2.off, n->e2.bs, 2 * w, H2, W2, B));
  NN_TRY(conv_bwd_weight<T>(n, L[2], A + n->p1.off, n->p1.bs, G + n->e2.off, n->e2.bs, B));
  NN_TRY(conv_bwd_data(n, L[2], G + n->e2.off, n->e2.bs, G + n->p1.off, n->p1.bs, B));
  // p1 = pool(s1)
  nn::k_pool_bwd<<<nn::nblk((int64_t)B * w * H * W), 256>>>(G + n->p1.off, n->p1.bs, G + n->s1.off, n->s1.bs, w, H, W, B);
  NN_CU(cudaGetLastError());
  // s1 = relu(conv(e1))
  NN_TRY(relu_mask<T>(G + n->s1.off, n->s1.bs, A + n->s1.off, n->s1.bs, w, H, W, B));
  NN_TRY(conv_bwd_weight<T>(n, L[1], A + n->e1.off, n->e1.bs, G + n->s1.off, n->s1.bs, B));
  NN_TRY(conv_bwd_data(n, L[1], G + n->s1.off, n->s1.bs, G + n->e1.off, n->e1.bs, B));
  // e1 = relu(conv(x))
  NN_TRY(relu_mask<T>(G + n->e1.off, n->e1.bs, A + n->e1.off, n->e1.bs, w, H, W, B));
  NN_TRY(conv_bwd_weight<T>(n, L[0], A + n->x_in.off, n->x_in.bs, G + n->e1.off, n->e1.bs, B));
  NN_CU(cudaDeviceSynchronize());
  return VLB_OK;
}

int refresh_compute_copy(vlb_nn *n) {
  if (n->storage != VLB_NN_BF16) return VLB_OK;
  nn::k_convert<__nv_bfloat16><<<nn::nblk(n->np), 256>>>(n->p, (__nv_bfloat16 *)n->pc, n->np);
  NN_CU(cudaGetLastError());
  return VLB_OK;
}

}  // namespace

extern "C" {

int vlb_nn_create(int32_t in_ch, int32_t out_ch, int32_t width, int32_t H, int32_t W, int32_t max_batch,
                  int32_t storage, uint64_t seed, vlb_nn **out) {
  if (!out) return vlb::set_error(VLB_EINVAL, "vlb_nn_create: out is NULL");
  *out = nullptr;
  if (in_ch < 1 || out_ch < 1 || width < 1 || H < 4 || W < 4 || (H % 4) || (W % 4) || max_batch < 1 ||
      (storage != VLB_NN_F32 && storage != VLB_NN_BF16))
    return vlb::set_error(VLB_EINVAL, "vlb_nn_create: bad shape (H and W must be multiples of 4) or storage");
  vlb_nn *n = new (std::nothrow) vlb_nn();
  if (!n) return vlb::set_error(VLB_ENOMEM, "vlb_nn_create: host allocation");
  n->ci = in_ch;
  n->co = out_ch;
  n->width = width;
  n->H = H;
  n->W = W;
  n->maxb = max_batch;
  n->storage = storage;
  const int w = width, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
  const int spec[11][5] = {{in_ch, w, 3, H, W},        {w, w, 3, H, W},          {w, 2 * w, 3, H2, W2},
                           {2 * w, 2 * w, 3, H2, W2},  {2 * w, 4 * w, 3, H4, W4}, {4 * w, 4 * w, 3, H4, W4},
                           {6 * w, 2 * w, 3, H2, W2},  {2 * w, 2 * w, 3, H2, W2}, {3 * w, w, 3, H, W},
                           {w, w, 3, H, W},            {w, out_ch, 1, H, W}};
  int64_t off = 0, wmax = 0, dwmax = 0;
  for (const auto &sp : spec) {
    NNLayer l{sp[0], sp[1], sp[2], sp[3], sp[4], 0, 0};
    l.woff = off;
    off += (int64_t)l.cin * l.cout * l.k * l.k;
    l.boff = off;
    off += l.cout;
    wmax = std::max<int64_t>(wmax, (int64_t)l.cin * l.cout * l.k * l.k);
    n->L.push_back(l);
  }
  dwmax = wmax;
  n->np = off;
  // activation layout per sample (elements), in one buffer with batch stride = per-sample total
  const int64_t HW = (int64_t)H * W, HW2 = (int64_t)H2 * W2, HW4 = (int64_t)H4 * W4;
  int64_t o = 0;
  auto take = [&](int64_t sz) {
    const int64_t r = o;
    o += sz;
    return r;
  };
  const int64_t x0 = take(in_ch * HW), e10 = take(w * HW), c10 = take(3 * w * HW), p10 = take(w * HW2),
                e20 = take(2 * w * HW2), c20 = take(6 * w * HW2), p20 = take(2 * w * HW4), e30 = take(4 * w * HW4),
                b30 = take(4 * w * HW4), d20 = take(2 * w * HW2), t20 = take(2 * w * HW2), d10 = take(w * HW),
                t10 = take(w * HW);
  const int64_t per = o;
  auto V = [&](int64_t off_) { return View{off_, per}; };
  n->x_in = V(x0);
  n->e1 = V(e10);
  n->c1 = V(c10);
  n->s1 = V(c10 + 2 * w * HW);   // s1 is the second slice of c1
  n->p1 = V(p10);
  n->e2 = V(e20);
  n->c2 = V(c20);
  n->s2 = V(c20 + 4 * w * HW2);  // s2 is the second slice of c2
  n->p2 = V(p20);
  n->e3 = V(e30);
  n->b3 = V(b30);
  n->d2 = V(d20);
  n->t2 = V(t20);
  n->d1 = V(d10);
  n->t1 = V(t10);
  n->act_n = per * max_batch;
  n->wt_n = wmax;
  n->dwp_n = dwmax * n->nsplit;
  const size_t es = storage == VLB_NN_BF16 ? 2 : 4;
  cudaError_t e = cudaMalloc(&n->p, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMalloc(&n->g, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMalloc(&n->m, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMalloc(&n->v, sizeof(float) * n->np);
  if (e == cudaSuccess && storage == VLB_NN_BF16) e = cudaMalloc(&n->pc, 2 * n->np);
  if (e == cudaSuccess) e = cudaMalloc(&n->act, es * n->act_n);
  if (e == cudaSuccess) e = cudaMalloc(&n->gr, sizeof(float) * n->act_n);
  if (e == cudaSuccess) e = cudaMalloc(&n->wt, sizeof(float) * n->wt_n);
  if (e == cudaSuccess) e = cudaMalloc(&n->dwp, sizeof(float) * n->dwp_n);
  if (e == cudaSuccess) e = cudaMalloc(&n->lossp, sizeof(double) * 1024);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->g, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->p, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->act, 0, es * n->act_n);
  for (size_t i = 0; i < n->L.size() && e == cudaSuccess; i++) {
    const NNLayer &l = n->L[i];
    const int64_t nw = (int64_t)l.cin * l.cout * l.k * l.k;
    const float bound = (float)std::sqrt(6.0 / ((double)l.cin * l.k * l.k));
    nn::k_init_params<<<nn::nblk(nw), 256>>>(n->p, l.woff, nw, bound, seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    vlb_nn_destroy(n);
    return vlb::set_error(e == cudaErrorMemoryAllocation ? VLB_ENOMEM : VLB_ECUDA, "vlb_nn_create: %s",
                          cudaGetErrorString(e));
  }
  const int rc = refresh_compute_copy(n);
  if (rc) {
    vlb_nn_destroy(n);
    return rc;
  }
  *out = n;
  return VLB_OK;
}

int vlb_nn_num_params(const vlb_nn *n, int64_t *np) {
  if (!n || !np) return vlb::set_error(VLB_EINVAL, "vlb_nn_num_params: NULL argument");
  *np = n->np;
  return VLB_OK;
}

int vlb_nn_get_params(const vlb_nn *n, float *host) {
  if (!n || !host) return vlb::set_error(VLB_EINVAL, "vlb_nn_get_params: NULL argument");
  NN_CU(cudaMemcpy(host, n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  return VLB_OK;
}

int vlb_nn_set_params(vlb_nn *n, const float *host) {
  if (!n || !host) return vlb::set_error(VLB_EINVAL, "vlb_nn_set_params: NULL argument");
  NN_CU(cudaMemcpy(n->p, host, sizeof(float) * n->np, cudaMemcpyHostToDevice));
  NN_TRY(refresh_compute_copy(n));
  NN_CU(cudaDeviceSynchronize());
  return VLB_OK;
}

int vlb_nn_set_tensor_cores(vlb_nn *n, int32_t enable) {
  if (!n) return vlb::set_error(VLB_EINVAL, "vlb_nn_set_tensor_cores: NULL net");
  n->tc = enable ? 1 : 0;
  return VLB_OK;
}

int vlb_nn_forward(vlb_nn *n, const float *d_x, float *d_y, int32_t batch) {
  if (!n || !d_x || !d_y || batch < 1 || batch > n->maxb)
    return vlb::set_error(VLB_EINVAL, "vlb_nn_forward: NULL argument or batch outside [1, max_batch]");
  return n->storage == VLB_NN_BF16 ? forward_t<__nv_bfloat16>(n, d_x, d_y, batch) : forward_t<float>(n, d_x, d_y, batch);
}

int vlb_nn_mse(vlb_nn *n, const float *d_y, const float *d_target, float *d_dy, int32_t batch, double *loss) {
  if (!n || !d_y || !d_target || !d_dy || !loss || batch < 1 || batch > n->maxb)
    return vlb::set_error(VLB_EINVAL, "vlb_nn_mse: NULL argument or bad batch");
  const int64_t cnt = (int64_t)batch * n->co * n->H * n->W;
  const int blocks = 1024;
  nn::k_mse<<<blocks, 256>>>(d_y, d_target, d_dy, cnt, n->lossp);
  NN_CU(cudaGetLastError());
  std::vector<double> h(blocks);
  NN_CU(cudaMemcpy(h.data(), n->lossp, sizeof(double) * blocks, cudaMemcpyDeviceToHost));
  double s = 0.0;
  for (double x : h) s += x;
  *loss = s / (double)cnt;
  return VLB_OK;
}

int vlb_nn_backward(vlb_nn *n, const float *d_dy, int32_t batch) {
  if (!n || !d_dy || batch < 1 || batch > n->maxb)
    return vlb::set_error(VLB_EINVAL, "vlb_nn_backward: NULL argument or bad batch");
  return n->storage == VLB_NN_BF16 ? backward_t<__nv_bfloat16>(n, d_dy, batch) : backward_t<float>(n, d_dy, batch);
}

int vlb_nn_get_grads(const vlb_nn *n, float *host) {
  if (!n || !host) return vlb::set_error(VLB_EINVAL, "vlb_nn_get_grads: NULL argument");
  NN_CU(cudaMemcpy(host, n->g, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  return VLB_OK;
}

int vlb_nn_adam(vlb_nn *n, float lr, float beta1, float beta2, float eps, int64_t t) {
  if (!n || t < 1) return vlb::set_error(VLB_EINVAL, "vlb_nn_adam: NULL net or t < 1");
  const float c1 = 1.0f - (float)std::pow((double)beta1, (double)t);
  const float c2 = 1.0f - (float)std::pow((double)beta2, (double)t);
  nn::k_adam<<<nn::nblk(n->np), 256>>>(n->p, n->g, n->m, n->v, n->np, lr, beta1, beta2, eps, c1, c2);
  NN_CU(cudaGetLastError());
  NN_TRY(refresh_compute_copy(n));
  NN_CU(cudaDeviceSynchronize());
  return VLB_OK;
}

void vlb_nn_destroy(vlb_nn *n) {
  if (!n) return;
  cudaDeviceSynchronize();
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  if (n->pc) cudaFree(n->pc);
  cudaFree(n->act);
  cudaFree(n->gr);
  cudaFree(n->wt);
  cudaFree(n->dwp);
  cudaFree(n->lossp);
  if (n->d_err) cudaFree(n->d_err);
  delete n;
}

}  // extern "C"

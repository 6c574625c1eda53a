// FP64 throughput probes: the denominator of the engine's roofline.
//
// The integral kernels are bound by the FP64 pipe, and the one FP64 figure a
// roofline needs is how fast this GPU retires FP64 multiply-adds. These
// kernels measure it directly, in the same process as the work they judge:
//  * kind 0: scalar DFMA, 8 independent dependency chains per thread;
//  * kind 1..3: the FP64 tensor-core instruction (DMMA, mma.sync .f64) in the
//    shapes m8n8k4, m16n8k4 and m16n8k16, 4 independent accumulators per warp.
// Operands are register-resident; nothing is read from memory in the loop. A
// result is stored only under a condition that never holds, so the work
// cannot be removed. FLOPs count 2 per multiply-add.
#include <cuda_runtime.h>

#include "../../include/mdx.h"

namespace {

constexpr int kProbeBlock = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kSink = 4096;

// target of the never-taken stores (a valid device address all the same)
__device__ double g_probe_sink[kSink];

__global__ void __launch_bounds__(kProbeBlock) k_probe_dfma(int iters, double* sink) {
  const double m = 0.9999999999, c = 1e-12;
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-9 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x % kSink] = s;
}

// one DMMA instruction of the given shape, accumulator d updated in place
template <int KIND>
__device__ __forceinline__ void dmma(double (&d)[4], const double (&a)[8], const double (&b)[4]) {
  if constexpr (KIND == 1) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a[0]), "d"(b[0]));
  } else if constexpr (KIND == 2) {
    asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(b[0]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
        "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
          "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
}

template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_probe_dmma(int iters, double* sink) {
  double a[8], b[4], d[4][4];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3 * (1 + ((threadIdx.x + k) & 7));
#pragma unroll
  for (int k = 0; k < 4; ++k) b[k] = 1e-3 * (1 + ((threadIdx.x + 3 * k) & 7));
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) d[j][k] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) dmma<KIND>(d[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) s += d[j][k];
  if (s == -1.0) sink[blockIdx.x % kSink] = s;
}

// FLOPs of one launch: per thread (DFMA) or per warp (DMMA) work x threads or warps
double probe_flops(int kind, int iters, int blocks) {
  const double threads = (double)blocks * kProbeBlock;
  if (kind == 0) return 2.0 * 8.0 * iters * threads;
  const double mnk = kind == 1 ? 8.0 * 8 * 4 : (kind == 2 ? 16.0 * 8 * 4 : 16.0 * 8 * 16);
  return 2.0 * mnk * 4.0 * iters * (threads / 32.0);
}

cudaError_t probe_launch(int kind, int iters, int blocks, double* sink, cudaStream_t s) {
  switch (kind) {
    case 0: k_probe_dfma<<<blocks, kProbeBlock, 0, s>>>(iters, sink); break;
    case 1: k_probe_dmma<1><<<blocks, kProbeBlock, 0, s>>>(iters, sink); break;
    case 2: k_probe_dmma<2><<<blocks, kProbeBlock, 0, s>>>(iters, sink); break;
    default: k_probe_dmma<3><<<blocks, kProbeBlock, 0, s>>>(iters, sink); break;
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" mdx_status mdx_fp64_peak(int kind, int reps, double* gflops, void* stream) {
  if (kind < 0 || kind > 3 || reps < 1 || !gflops) return MDX_EINVAL;
  *gflops = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  const int blocks = sms * kBlocksPerSm;
  // about 100 ms per launch at ~1.2 TFLOP/s (the DMMA loops do more work per iteration)
  const int iters = kind == 0 ? 24576 : (kind == 3 ? 1024 : (kind == 2 ? 4096 : 8192));
  double* sink = nullptr;   // never written: the store's condition never holds
  if (cudaGetSymbolAddress((void**)&sink, g_probe_sink) != cudaSuccess) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return MDX_ECUDA;
  }
  cudaError_t e = probe_launch(kind, iters, blocks, sink, s);   // warm-up (clocks, instruction cache)
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = probe_launch(kind, iters, blocks, sink, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.0f) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  *gflops = probe_flops(kind, iters, blocks) * reps / (ms * 1e-3) * 1e-9;
  return MDX_OK;
}

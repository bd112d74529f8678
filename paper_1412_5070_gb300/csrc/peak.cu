// peak.cu -- arithmetic peaks of the device, measured in place: the
// denominators of the library's roofline figures.  Measurement aid with no
// counterpart in the paper.
//
// Every kernel runs independent chains of one instruction in a loop, sized to
// a few hundred milliseconds, on SMs x 8 blocks of 256 threads; one warm-up
// launch, then CUDA events around one launch.  Flops counted: 2 per FMA, and
// 2 m n k per matrix multiply-accumulate of shape m x n x k.
#include <cuda_runtime.h>

#include "../../include/f12int.h"

namespace {

constexpr int kChains = 8;

template <class T>
__global__ void peak_fma(T *out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x * 1e-3 + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 matrix multiply-accumulate (the DMMA path of mma.sync) with four
// independent accumulators per warp.  SHAPE 0: m8n8k4, 1: m16n8k4, 2: m16n8k16.
template <int SHAPE>
__global__ void peak_dmma(double *out, int iters) {
  const double a = threadIdx.x * 1e-6, b = 1.0 - threadIdx.x * 1e-7;
  double c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[j][q] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if constexpr (SHAPE == 0) {
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c[j][0]), "+d"(c[j][1])
                     : "d"(a), "d"(b));
      } else if constexpr (SHAPE == 1) {
        asm volatile(
            "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
            : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
            : "d"(a), "d"(a), "d"(b));
      } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
            "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
            : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
            : "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(b), "d"(b), "d"(b), "d"(b));
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += c[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// flops of one warp-wide instruction of the kind
double flops_per_warp_inst(int kind) {
  switch (kind) {
    case 0: return 2.0 * 32;                // DFMA, 32 lanes
    case 1: return 2.0 * 8 * 8 * 4;        // m8n8k4
    case 2: return 2.0 * 16 * 8 * 4;       // m16n8k4
    case 3: return 2.0 * 16 * 8 * 16;      // m16n8k16
    case 4: return 2.0 * 32;                // FFMA
    default: return 0.0;
  }
}

template <class F>
int time_launch(F launch, float *ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return F12INT_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return F12INT_ECUDA;
  }
  launch(true);   // warm-up
  cudaEventRecord(e0);
  launch(false);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? F12INT_OK : F12INT_ECUDA;
}

}  // namespace

extern "C" int f12int_measure_peak(int device, int kind, double *tflops) {
  if (!tflops || kind < 0 || kind > 4) return F12INT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return F12INT_ECUDA;
  if (device < 0 || device >= ndev) return F12INT_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return F12INT_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256;
  void *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) {
    cudaSetDevice(prev);
    return F12INT_ENOMEM;
  }
  // iterations per launch: a few hundred milliseconds at the expected rates
  int iters = 1;
  int64_t insts_per_iter = 0;   // warp instructions per loop iteration and warp
  switch (kind) {
    case 0: iters = 20000; insts_per_iter = kChains; break;
    case 1: case 2: case 3: iters = kind == 3 ? 500 : 2000; insts_per_iter = 4; break;
    case 4: iters = 200000; insts_per_iter = kChains; break;
  }
  float ms = 0.f;
  int rc = time_launch(
      [&](bool warm) {
        const int it = warm ? iters / 20 + 1 : iters;
        switch (kind) {
          case 0: peak_fma<double><<<blocks, threads>>>((double *)out, it, 0.999, 1e-3); break;
          case 1: peak_dmma<0><<<blocks, threads>>>((double *)out, it); break;
          case 2: peak_dmma<1><<<blocks, threads>>>((double *)out, it); break;
          case 3: peak_dmma<2><<<blocks, threads>>>((double *)out, it); break;
          case 4: peak_fma<float><<<blocks, threads>>>((float *)out, it, 0.999f, 1e-3f); break;
        }
      },
      &ms);
  cudaFree(out);
  cudaSetDevice(prev);
  if (rc != F12INT_OK) return rc;
  const double warps = (double)blocks * threads / 32.0;
  *tflops = flops_per_warp_inst(kind) * (double)insts_per_iter * iters * warps / (ms * 1e-3) / 1e12;
  return F12INT_OK;
}

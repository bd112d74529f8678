// fma_peak.cu -- FP64 / FP32 fused multiply-add throughput of the device:
// 8 independent FMA chains per thread, SMs x 8 blocks of 256 threads, timed
// with CUDA events after one warm-up launch.  Corroborates the FP64 rate the
// bench's roofline uses (152 SMs x 2 FP64 FMA per clock x 2 flops x clock).
#include <cstdio>
#include <cuda_runtime.h>

template <class T>
__global__ void fma_chains(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
    x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
static double tflops(int blocks, int threads, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  fma_chains<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)1e-3);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-3);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  printf("SMs %d\n", sms);
  for (int rep = 0; rep < 2; ++rep) {
    printf("fp64 TFLOP/s %.3f\n", tflops<double>(sms * 8, 256, 20000));
    printf("fp32 TFLOP/s %.3f\n", tflops<float>(sms * 8, 256, 100000));
  }
  return 0;
}

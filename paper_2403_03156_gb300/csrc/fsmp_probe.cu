// fsmp_probe.cu -- microbenchmarks for the roofline denominators of the chain kernels:
// shared-memory load bandwidth (the bound of the FP32 chain kernel) and the FP64 / FP32 FMA
// rates (the bound of the FP64 chain kernel on a part with a reduced FP64 rate). Each is
// timed with CUDA events on a private stream after a warm-up launch.
#include "fsmp_internal.h"

namespace fsmp {
namespace {

// Every thread streams float4 loads from a 32 KiB shared buffer (conflict-free: consecutive
// lanes read consecutive 16-byte words) and folds them into a register sum.
__global__ void __launch_bounds__(256) smem_read_kernel(float* sink, int iters) {
  __shared__ float4 buf[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) buf[i] = make_float4(i, i + 1, i + 2, i + 3);
  __syncthreads();
  float4 acc = make_float4(0, 0, 0, 0);
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float4 v = buf[(idx + k * 256) & 2047];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    idx = (idx + 32) & 2047;
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.0f) sink[0] = acc.x;
}

template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(T* sink, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == (T)-12345) sink[0] = x0;
}

}  // namespace

cudaError_t measure_peaks(int sm_count, double* smem_gbs, double* fp64_tflops, double* fp32_tflops) {
  cudaStream_t st;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  float* sink = nullptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  e = cudaMalloc(&sink, 64);
  float ms = 0.f;
  if (e == cudaSuccess) {
    const int blocks = sm_count * 4, thr = 256;
    const int it_s = 4000;
    smem_read_kernel<<<blocks, thr, 0, st>>>(sink, 100);
    cudaEventRecord(e0, st);
    smem_read_kernel<<<blocks, thr, 0, st>>>(sink, it_s);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *smem_gbs = (double)blocks * thr * it_s * 8 * 16 / (ms * 1e-3) / 1e9;
    const int it_d = 400;
    fma_kernel<double><<<blocks, thr, 0, st>>>((double*)sink, 10, 0.999, 0.001);
    cudaEventRecord(e0, st);
    fma_kernel<double><<<blocks, thr, 0, st>>>((double*)sink, it_d, 0.999, 0.001);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *fp64_tflops = 2.0 * blocks * thr * it_d * 64 / (ms * 1e-3) / 1e12;
    const int it_f = 8000;
    fma_kernel<float><<<blocks, thr, 0, st>>>(sink, 10, 0.999f, 0.001f);
    cudaEventRecord(e0, st);
    fma_kernel<float><<<blocks, thr, 0, st>>>(sink, it_f, 0.999f, 0.001f);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *fp32_tflops = 2.0 * blocks * thr * it_f * 64 / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  cudaFree(sink);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return e;
}

}  // namespace fsmp

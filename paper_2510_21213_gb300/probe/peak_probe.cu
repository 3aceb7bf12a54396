// Throughput probe of the GPU: FP64 FMA (SIMT), FP32 FMA (SIMT), FP64 DMMA
// (mma.sync m8n8k4) and an HBM copy, timed with CUDA events. Gives the ALU
// roofline denominators for the FP64 and FP32 kernels of this library.
// Build and run: python -m paper_2510_21213_gb300.probe.run_probe
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345.678) out[blockIdx.x] = s;
}
__global__ void dmma_kernel(double* out, int iters) {
  double a = threadIdx.x * 1e-3, b = 1.0 + threadIdx.x * 1e-4;
  double c0 = 0, c1 = 0, d0 = 0, d1 = 0, e0 = 0, e1 = 0, f0 = 0, f1 = 0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(e0), "+d"(e1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(f0), "+d"(f1) : "d"(a), "d"(b));
    }
  }
  double s = c0 + c1 + d0 + d1 + e0 + e1 + f0 + f1;
  if (s == 12345.678) out[blockIdx.x] = s;
}
__global__ void copy_kernel(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}
int main() {
  int dev = 0; cudaDeviceProp prop; cudaGetDeviceProperties(&prop, dev);
  printf("device %s SMs %d cc %d.%d\n", prop.name, prop.multiProcessorCount, prop.major, prop.minor);
  int sms = prop.multiProcessorCount;
  double* outd; cudaMalloc(&outd, 1 << 20);
  float* outf; cudaMalloc(&outf, 1 << 20);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  int blocks = sms * 8, threads = 256;
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 4096;
    cudaEventRecord(e0);
    fma_kernel<double><<<blocks, threads>>>(outd, iters, 0.999, 1e-3);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 64 * iters * (double)blocks * threads;
    printf("FP64 FMA: %.3f ms  %.3f TFLOP/s\n", ms, flops / ms / 1e9);
    iters = 65536;
    cudaEventRecord(e0);
    fma_kernel<float><<<blocks, threads>>>(outf, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    flops = 2.0 * 64 * iters * (double)blocks * threads;
    printf("FP32 FMA: %.3f ms  %.3f TFLOP/s\n", ms, flops / ms / 1e9);
    iters = 1024;
    cudaEventRecord(e0);
    dmma_kernel<<<blocks, threads>>>(outd, iters);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    // each mma m8n8k4 per warp = 8*8*4*2 flops
    flops = 16.0 * iters * (double)blocks * (threads / 32) * 512;
    printf("FP64 DMMA: %.3f ms  %.3f TFLOP/s  err=%s\n", ms, flops / ms / 1e9, cudaGetErrorString(cudaGetLastError()));
  }
  size_t n = (size_t)1 << 28;  // 4 GiB of float4? n float4 = 16 B each -> 4 GiB
  float4 *a, *b; cudaMalloc(&a, n * 16); cudaMalloc(&b, n * 16);
  cudaMemset(a, 0, n * 16);
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    copy_kernel<<<sms * 16, 512>>>(a, b, n);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("copy: %.3f ms %.1f GB/s\n", ms, 2.0 * n * 16 / ms / 1e6);
  }
  printf("final err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}

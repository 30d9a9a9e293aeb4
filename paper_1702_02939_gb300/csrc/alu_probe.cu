// Standalone arithmetic-throughput microbenchmark (FP64 / FP32 / INT pipes).
// Not part of libcellgb.so.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_probe alu_probe.cu && ./alu_probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int ITERS>
__global__ void k_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <int ITERS>
__global__ void k_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <int ITERS>
__global__ void k_imad(uint32_t* out, uint32_t a, uint32_t b) {
  uint32_t x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <int ITERS>
__global__ void k_mul64hi(uint64_t* out, uint64_t a) {
  uint64_t x0 = threadIdx.x + 11, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) {
    x0 = __umul64hi(x0, a) ^ (x0 * a); x1 = __umul64hi(x1, a) ^ (x1 * a);
    x2 = __umul64hi(x2, a) ^ (x2 * a); x3 = __umul64hi(x3, a) ^ (x3 * a);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int ITERS>
__global__ void k_drcp(double* out, double a) {
  double x0 = threadIdx.x + 1.5, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) {
    x0 = a / x0 + 1.0; x1 = a / x1 + 1.0; x2 = a / x2 + 1.0; x3 = a / x3 + 1.0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int ITERS>
__global__ void k_dsqrt(double* out, double a) {
  double x0 = threadIdx.x + 1.5, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS; ++i) {
    x0 = sqrt(x0) + a; x1 = sqrt(x1) + a; x2 = sqrt(x2) + a; x3 = sqrt(x3) + a;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
template <int ITERS>
__global__ void k_dlogcos(double* out, double a) {
  double x0 = threadIdx.x * 1e-4 + 0.5, x1 = x0 + 0.1;
  for (int i = 0; i < ITERS; ++i) {
    x0 = log(x0 + 1.0) * cos(x0) + a; x1 = log(x1 + 1.0) * cos(x1) + a;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1;
}

int main() {
  int dev = 0; CK(cudaSetDevice(dev));
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int sms = p.multiProcessorCount, l2 = 0, clk = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("name %s sms %d l2 %d bytes smem/block optin %zu regs/sm %d clock_khz %d cc %d.%d\n", p.name, sms, l2,
         p.sharedMemPerBlockOptin, p.regsPerMultiprocessor, clk, p.major, p.minor);
  const int threads = 256, blocks = sms * 8;
  const size_t nthreads = (size_t)threads * blocks;
  void* buf; CK(cudaMalloc(&buf, nthreads * 8));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  auto report = [&](const char* name, double ops) {
    cudaEventElapsedTime(&ms, e0, e1);
    double rate = ops / (ms * 1e-3);
    printf("%-10s %8.3f ms  %10.3f Gop/s  %8.2f op/clk/SM (at %.0f MHz nominal)\n", name, ms, rate * 1e-9,
           rate / (sms * (clk * 1e3)), clk / 1e3);
  };
  const int IT = 4096;
  for (int rep = 0; rep < 2; ++rep) {
    k_dfma<IT><<<blocks, threads>>>((double*)buf, 0.999, 1e-3);
    CK(cudaEventRecord(e0)); k_dfma<IT><<<blocks, threads>>>((double*)buf, 0.999, 1e-3); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("dfma", (double)nthreads * IT * 8);
    CK(cudaEventRecord(e0)); k_ffma<IT * 8><<<blocks, threads>>>((float*)buf, 0.999f, 1e-3f); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("ffma", (double)nthreads * IT * 8 * 8);
    CK(cudaEventRecord(e0)); k_imad<IT * 8><<<blocks, threads>>>((uint32_t*)buf, 1664525u, 1013904223u); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("imad", (double)nthreads * IT * 8 * 8);
    CK(cudaEventRecord(e0)); k_mul64hi<IT><<<blocks, threads>>>((uint64_t*)buf, 0x9E3779B97F4A7C15ull); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("mul64", (double)nthreads * IT * 4);
    CK(cudaEventRecord(e0)); k_drcp<IT / 4><<<blocks, threads>>>((double*)buf, 0.5); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("ddiv", (double)nthreads * IT / 4 * 4);
    CK(cudaEventRecord(e0)); k_dsqrt<IT / 4><<<blocks, threads>>>((double*)buf, 0.5); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("dsqrt", (double)nthreads * IT / 4 * 4);
    CK(cudaEventRecord(e0)); k_dlogcos<IT / 16><<<blocks, threads>>>((double*)buf, 0.1); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); report("dlog+cos", (double)nthreads * IT / 16 * 2);
  }
  CK(cudaGetLastError());
  CK(cudaFree(buf));
  return 0;
}

// peak_probe.cu -- measures the FP64 and FP32 FMA throughput and a copy
// bandwidth of the current GPU (the FP64 rate is the roofline denominator of
// the FP64-bound kernels; it is not in the driver's measured-peaks file).
// Prints one JSON line.  Built and run by `python bench.py --peak-probe`.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int k = 0; k < iters; ++k) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void copy_k(const double2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) { printf("{\"error\": \"no device\"}\n"); return 1; }
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  void* out = nullptr;
  cudaMalloc(&out, (size_t)blocks * threads * 8);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double tf64 = 0, tf32 = 0, gbs = 0;
  for (int rep = 0; rep < 2; ++rep) {
    const int it64 = 4096, it32 = 65536;
    float ms = 0;
    fma_loop<double><<<blocks, threads>>>((double*)out, it64, 0.999, 1e-3);
    cudaEventRecord(e0);
    fma_loop<double><<<blocks, threads>>>((double*)out, it64, 0.999, 1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    tf64 = 2.0 * 8 * it64 * (double)blocks * threads / ms / 1e9;
    fma_loop<float><<<blocks, threads>>>((float*)out, it32, 0.999f, 1e-3f);
    cudaEventRecord(e0);
    fma_loop<float><<<blocks, threads>>>((float*)out, it32, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    tf32 = 2.0 * 8 * it32 * (double)blocks * threads / ms / 1e9;
  }
  const size_t n2 = (size_t)1 << 27;  // 128 Mi double2 = 2 GiB per buffer
  double2 *a = nullptr, *b = nullptr;
  if (cudaMalloc(&a, n2 * 16) == cudaSuccess && cudaMalloc(&b, n2 * 16) == cudaSuccess) {
    cudaMemset(a, 0, n2 * 16);
    for (int rep = 0; rep < 3; ++rep) {
      float ms = 0;
      cudaEventRecord(e0);
      copy_k<<<p.multiProcessorCount * 16, 256>>>(a, b, n2);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      const double g = 2.0 * n2 * 16 / ms / 1e6;
      if (g > gbs) gbs = g;
    }
  }
  printf("{\"gpu\": \"%s\", \"sms\": %d, \"fp64_tflops\": %.4f, \"fp32_tflops\": %.3f, \"copy_gbs\": %.1f, \"error\": \"%s\"}\n",
         p.name, p.multiProcessorCount, tf64, tf32, gbs, cudaGetErrorString(cudaGetLastError()));
  return 0;
}

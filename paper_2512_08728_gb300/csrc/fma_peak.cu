// Throughput probe for the rooflines of the FP64 kernels: dependent-chain FMA throughput in
// FP64 and FP32 over the whole GPU, and streaming read bandwidth with one FP64 operation
// per loaded element (the arithmetic intensity of a block operator application).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_peak fma_peak.cu
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { \
  printf("CUDA error %s at line %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); exit(1); } } while (0)

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
    x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345.678) out[0] = s;   // keeps the chains live
}

__global__ void read_fma_f64(const double2* __restrict__ x, size_t n2, double* out) {
  double s0 = 0, s1 = 0;
  const double c = 1.000001;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = __ldg(x + i);
    s0 = fma(v.x, c, s0);
    s1 = fma(v.y, c, s1);
  }
  if (s0 + s1 == 12345.678) out[0] = s0;
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  printf("device %s, %d SMs\n", p.name, p.multiProcessorCount);
  double* out;
  CK(cudaMalloc(&out, 64));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const dim3 g(p.multiProcessorCount * 8), b(256);
  float ms;
  for (int rep = 0; rep < 2; rep++) {
    fma_chains<double><<<g, b>>>(out, 4096, 1.0000001, 1e-9);
    CK(cudaEventRecord(e0));
    fma_chains<double><<<g, b>>>(out, 4096, 1.0000001, 1e-9);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("FP64 FMA: %.3f TFLOP/s\n", 2.0 * 8 * 4096 * (double)g.x * b.x / ms * 1e-9);
    fma_chains<float><<<g, b>>>((float*)out, 65536, 1.0000001f, 1e-9f);
    CK(cudaEventRecord(e0));
    fma_chains<float><<<g, b>>>((float*)out, 65536, 1.0000001f, 1e-9f);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("FP32 FMA: %.3f TFLOP/s\n", 2.0 * 8 * 65536 * (double)g.x * b.x / ms * 1e-9);
  }
  const size_t bytes = (size_t)2 << 30;
  void* buf;
  CK(cudaMalloc(&buf, bytes));
  CK(cudaMemset(buf, 0, bytes));
  for (int bpsm = 4; bpsm <= 16; bpsm *= 2) {
    const dim3 gg(p.multiProcessorCount * bpsm);
    for (int w = 0; w < 2; w++) {
      CK(cudaEventRecord(e0));
      read_fma_f64<<<gg, b>>>((const double2*)buf, bytes / 16, out);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
    }
    printf("stream FP64 read + 1 FMA/element, %d blocks/SM: %.1f GB/s\n", bpsm, bytes / ms * 1e-6);
  }
  CK(cudaFree(buf));
  return 0;
}

// Grid-barrier latency microbenchmark (stand-alone program, not part of libkcmg): one
// cooperative kernel with one block of 320 threads per SM passes 20,000 grid barriers of
// three designs and reports microseconds per barrier from the GPU global timer.
//   A  one counter: fetch_add (acq_rel), then poll the counter for the generation target
//      (the barrier of the persistent coarse cycle);
//   B  a counter plus a separate generation flag released by the last block;
//   C  two levels: groups of G blocks on their own counters, then a root counter.
// Every spin is bounded; a timeout sets an error flag that the host reports.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 barrier_probe.cu
#include <cuda/atomic>
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ unsigned long long gtime() { unsigned long long t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t; }

// A: fetch_add + poll counter target
__device__ bool barA(unsigned int* cnt, int* err, unsigned int& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(*cnt);
    const unsigned int target = (gen + 1) * gridDim.x;
    unsigned int old = c.fetch_add(1u, cuda::memory_order_acq_rel);
    int o = 1;
    if (old + 1 != target) {
      long long s = 0;
      while (c.load(cuda::memory_order_acquire) < target) { if (++s > (1 << 22)) { *err = 1; o = 0; break; } }
    }
    ok = o;
  }
  ++gen;
  __syncthreads();
  return ok;
}
// B: counter + generation flag on separate lines; last arriver resets counter and bumps the flag
__device__ bool barB(unsigned int* cnt, unsigned int* flag, int* err, unsigned int& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(*cnt), f(*flag);
    int o = 1;
    if (c.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
      c.store(0u, cuda::memory_order_relaxed);
      f.store(gen + 1, cuda::memory_order_release);
    } else {
      long long s = 0;
      while (f.load(cuda::memory_order_acquire) != gen + 1) { if (++s > (1 << 22)) { *err = 1; o = 0; break; } }
    }
    ok = o;
  }
  ++gen;
  __syncthreads();
  return ok;
}
// C: two-level: groups of G blocks on their own counter lines (128 B apart), group leaders on a root counter, flag release
template <int G>
__device__ bool barC(unsigned int* sub, unsigned int* root, unsigned int* flag, int* err, unsigned int& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int grp = blockIdx.x / G;
    const int ngrp = (gridDim.x + G - 1) / G;
    const int gsize = min(G, (int)gridDim.x - grp * G);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> s_(sub[grp * 32]), r_(*root), f(*flag);
    int o = 1;
    bool release = false;
    if (s_.fetch_add(1u, cuda::memory_order_acq_rel) == (unsigned)gsize - 1) {
      s_.store(0u, cuda::memory_order_relaxed);
      if (r_.fetch_add(1u, cuda::memory_order_acq_rel) == (unsigned)ngrp - 1) {
        r_.store(0u, cuda::memory_order_relaxed);
        f.store(gen + 1, cuda::memory_order_release);
        release = true;
      }
    }
    if (!release) {
      long long s = 0;
      while (f.load(cuda::memory_order_acquire) != gen + 1) { if (++s > (1 << 22)) { *err = 1; o = 0; break; } }
    }
    ok = o;
  }
  ++gen;
  __syncthreads();
  return ok;
}

__global__ void kprobe(int variant, int iters, unsigned int* cnt, unsigned int* flag, unsigned int* sub, int* err, unsigned long long* out) {
  unsigned int gen = 0;
  unsigned long long t0 = gtime();
  for (int i = 0; i < iters; ++i) {
    bool ok;
    if (variant == 0) ok = barA(cnt, err, gen);
    else if (variant == 1) ok = barB(cnt, flag, err, gen);
    else if (variant == 2) ok = barC<8>(sub, cnt, flag, err, gen);
    else ok = barC<16>(sub, cnt, flag, err, gen);
    if (!ok) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = gtime() - t0;
}

int main() {
  int nsm; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  unsigned int *cnt, *flag, *sub; int* err; unsigned long long* out;
  cudaMalloc(&cnt, 4096); cudaMalloc(&flag, 4096); cudaMalloc(&sub, 64 * 32 * 4); cudaMalloc(&err, 4); cudaMalloc(&out, 8);
  const char* names[] = {"A fetch_add+poll counter", "B counter+flag", "C two-level G=8", "C two-level G=16"};
  for (int v = 0; v < 4; ++v) {
    for (int rep = 0; rep < 2; ++rep) {
      cudaMemset(cnt, 0, 4096); cudaMemset(flag, 0, 4096); cudaMemset(sub, 0, 64 * 32 * 4); cudaMemset(err, 0, 4);
      int iters = 20000;
      void* args[] = {&v, &iters, &cnt, &flag, &sub, &err, &out};
      cudaError_t e = cudaLaunchCooperativeKernel((void*)kprobe, nsm, 320, args, 0, 0);
      cudaError_t e2 = cudaDeviceSynchronize();
      unsigned long long ns = 0; int herr = 0;
      cudaMemcpy(&ns, out, 8, cudaMemcpyDeviceToHost); cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
      printf("%-26s grid %d: %.3f us/barrier (err %d, launch %s, sync %s)\n", names[v], nsm, ns / 1e3 / iters, herr,
             cudaGetErrorString(e), cudaGetErrorString(e2));
      if (e != cudaSuccess || e2 != cudaSuccess || herr) return 1;
    }
  }
  return 0;
}

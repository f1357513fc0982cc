// Kernel launch helper.  Every kernel of the library is a functor
//   struct K { __host__ __device__ void operator()(const KExec& ex, int block) const; };
// run with one CTA per block index; ex.tid / ex.nt are the thread index and
// count, ex.smem the dynamic shared memory, ex.sync() the CTA barrier.
#pragma once
#include "common.h"
#include <atomic>

#ifdef __CUDACC__
#define VB_HD __host__ __device__
#else
#define VB_HD
#endif

namespace vb {

extern std::atomic<int64_t> g_launches;   // kernels launched by the library

struct KExec {
  int tid, nt;
  double* smem;
#ifdef __CUDA_ARCH__
  __device__ void sync() const { __syncthreads(); }
#else
  VB_HD void sync() const {}
#endif
};

#ifdef __CUDACC__
template <class F>
__global__ void k_run(const F f) {
  extern __shared__ __align__(16) double vb_smem[];
  f(KExec{(int)threadIdx.x, (int)blockDim.x, vb_smem}, (int)blockIdx.x);
}

// the same with 256 threads and at least MINB resident CTAs per SM (the
// compiler caps the registers accordingly)
template <class F, int MINB>
__global__ void __launch_bounds__(256, MINB) k_run_lb(const F f) {
  extern __shared__ __align__(16) double vb_smem[];
  f(KExec{(int)threadIdx.x, (int)blockDim.x, vb_smem}, (int)blockIdx.x);
}

template <int MINB, class F>
inline void launch_lb(const F& f, int64_t nblocks, size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return;
  VB_CHECK(nblocks < (int64_t)INT32_MAX, VEM_EINVAL, "grid too large");
  if (smem > 48 * 1024)
    VB_CUDA(cudaFuncSetAttribute(k_run_lb<F, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_run_lb<F, MINB><<<(unsigned)nblocks, 256, smem, s>>>(f);
  VB_KERNEL_CHECK();
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// the same with 128 threads and at least MINB resident CTAs per SM
template <class F, int MINB>
__global__ void __launch_bounds__(128, MINB) k_run_lb128(const F f) {
  extern __shared__ __align__(16) double vb_smem[];
  f(KExec{(int)threadIdx.x, (int)blockDim.x, vb_smem}, (int)blockIdx.x);
}

template <int MINB, class F>
inline void launch_lb128(const F& f, int64_t nblocks, size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return;
  VB_CHECK(nblocks < (int64_t)INT32_MAX, VEM_EINVAL, "grid too large");
  if (smem > 48 * 1024)
    VB_CUDA(cudaFuncSetAttribute(k_run_lb128<F, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_run_lb128<F, MINB><<<(unsigned)nblocks, 128, smem, s>>>(f);
  VB_KERNEL_CHECK();
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// the same with up to MAXT threads per CTA (the compiler caps the registers
// so that a CTA of MAXT threads fits on an SM)
template <class F, int MAXT>
__global__ void __launch_bounds__(MAXT) k_run_mt(const F f) {
  extern __shared__ __align__(16) double vb_smem[];
  f(KExec{(int)threadIdx.x, (int)blockDim.x, vb_smem}, (int)blockIdx.x);
}

template <int MAXT, class F>
inline void launch_mt(const F& f, int64_t nblocks, int nthreads, size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return;
  VB_CHECK(nblocks < (int64_t)INT32_MAX, VEM_EINVAL, "grid too large");
  VB_CHECK(nthreads <= MAXT, VEM_EINVAL, "launch: more threads than the kernel's bound");
  if (smem > 48 * 1024)
    VB_CUDA(cudaFuncSetAttribute(k_run_mt<F, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_run_mt<F, MAXT><<<(unsigned)nblocks, nthreads, smem, s>>>(f);
  VB_KERNEL_CHECK();
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <class F>
inline void launch(const F& f, int64_t nblocks, int nthreads, size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return;
  VB_CHECK(nblocks < (int64_t)INT32_MAX, VEM_EINVAL, "grid too large");
  if (smem > 48 * 1024)
    VB_CUDA(cudaFuncSetAttribute(k_run<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_run<F><<<(unsigned)nblocks, nthreads, smem, s>>>(f);
  VB_KERNEL_CHECK();
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
#endif

VB_HD inline void flag_error(int* p, int v) {
#ifdef __CUDA_ARCH__
  atomicMax(p, v);
#else
  if (*p < v) *p = v;
#endif
}

// block-wide sum of one double per thread (deterministic tree), result valid in all threads
VB_HD inline double block_sum(const KExec& ex, double v, double* red) {
  red[ex.tid] = v;
  ex.sync();
  for (int s = 1; s < ex.nt; s <<= 1) {
    if ((ex.tid & (2 * s - 1)) == 0 && ex.tid + s < ex.nt) red[ex.tid] += red[ex.tid + s];
    ex.sync();
  }
  double r = red[0];
  ex.sync();
  return r;
}

}  // namespace vb

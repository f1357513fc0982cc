// Shared helpers of the vembddc library: status handling, device buffers,
// scaled-monomial index arithmetic (host and device).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <stdexcept>

#include "../../include/vembddc.h"

namespace vb {

// ---- errors: library code throws vb::Error; the C entry points catch it,
// ---- record the message and return the status.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

void set_last_error(const std::string& m);
extern thread_local std::string g_last_error;

#define VB_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::vb::Error(VEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define VB_CHECK(cond, status, msg)                     \
  do {                                                  \
    if (!(cond)) throw ::vb::Error((status), (msg));    \
  } while (0)

#define VB_KERNEL_CHECK() VB_CUDA(cudaGetLastError())

// ---- owning device buffer
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      (void)cudaGetLastError();
      throw Error(VEM_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void upload(const std::vector<T>& h, cudaStream_t s = 0) {
    if (h.size() != n) alloc(h.size());
    if (n) VB_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s = 0) {
    if (n) VB_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  std::vector<T> download(cudaStream_t s = 0) const {
    std::vector<T> h(n);
    if (n) {
      VB_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
      VB_CUDA(cudaStreamSynchronize(s));
    }
    return h;
  }
};

// ---- scaled monomials in graded order: degree, then first exponent
// ---- descending, then second exponent descending.
__host__ __device__ constexpr int pdim3(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
__host__ __device__ constexpr int pdim2(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) / 2; }
__host__ __device__ inline int idx3(int a, int b, int c) {
  int d = a + b + c;
  return pdim3(d - 1) + (d - a) * (d - a + 1) / 2 + (d - a - b);
}
__host__ __device__ inline int idx2(int a, int b) {
  int d = a + b;
  return pdim2(d - 1) + (d - a);
}
// exponents of the 3D monomial number i (i < pdim3(12)); host/device tables
struct Exp3 { unsigned char a, b, c, d; };
struct Exp2 { unsigned char a, b, d, pad; };
constexpr int kMaxMono3 = 455;   // pdim3(12)
constexpr int kMaxMono2 = 91;    // pdim2(12)

// counts of the element-interior DOFs
__host__ __device__ constexpr int n_d4(int k) { return 3 * pdim3(k - 3) - pdim3(k - 4); }
__host__ __device__ constexpr int n_d5(int k) { return pdim3(k - 1) - 1; }

// Gauss-Legendre rule on [0,1] with n points (Newton on P_n), host side.
void gauss01(int n, std::vector<double>& x, std::vector<double>& w);
void gauss01(int n, double* x, double* w);   // the same rule into caller-owned arrays
// interior Gauss-Lobatto nodes on [0,1] for degree k (k-1 nodes), host side
std::vector<double> lobatto_interior(int k);

}  // namespace vb

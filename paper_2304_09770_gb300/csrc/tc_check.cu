// Diagnostics of the tensor-core tile product used by the FP32 front
// factorization (tcgen05, three-part TF32 split, FP32 accumulation in TMEM):
// one 128 x 128 x 32 product on deterministic data against an FP64 product.
#include "common.h"
#include "launch.h"
#include "tc.cuh"

namespace vb {

// deterministic values in [-1, 1) with full FP32 mantissas
__device__ inline float tc_check_val(int m, int k, int which) {
  uint32_t h = (uint32_t)(m * 73856093) ^ (uint32_t)(k * 19349663) ^ (uint32_t)(which * 83492791);
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  return (float)((double)(h & 0xFFFFFFu) / (double)0x800000 - 1.0);
}

struct KTcCheck {
  double* out;   // [0] max |D - ref|, [1] max |ref|, [2] 1 if the product ran
  int* status;
  __device__ void operator()(const KExec& ex, int) const {
    TcCtx c;
    c.tiles = reinterpret_cast<float*>(ex.smem);
    c.mbar = reinterpret_cast<uint64_t*>(c.tiles + 2 * TC_PARTS * TC_TILE_FLOATS);
    c.taddr_slot = reinterpret_cast<uint32_t*>(c.mbar + 1);
    c.status = status;
    tc_init(ex, c);
    for (int q = ex.tid; q < TC_M * TC_K; q += ex.nt) {
      const int col = q / TC_M, mm = q % TC_M, o = tc_off(mm, col);
      tc_split3(tc_check_val(mm, col, 0), c.tiles, o);
      tc_split3(tc_check_val(mm, col, 1), c.tiles + TC_PARTS * TC_TILE_FLOATS, o);
    }
    double err = 0.0, mx = 0.0;
    const bool ran = tc_product(ex, c);
    if (ran) {
      const int w = ex.tid >> 5, lane = ex.tid & 31, rowblk = w & 3, colhalf = w >> 2;
      const int i = rowblk * 32 + lane;
      for (int cc = 0; cc < 2; ++cc) {
        float v[32];
        tc_ld32(c.taddr + ((uint32_t)(rowblk * 32) << 16) + (uint32_t)(colhalf * 64 + cc * 32), v);
        for (int q = 0; q < 32; ++q) {
          const int n = colhalf * 64 + cc * 32 + q;
          double ref = 0.0;
          for (int k = 0; k < TC_K; ++k) ref += (double)tc_check_val(i, k, 0) * (double)tc_check_val(n, k, 1);
          err = fmax(err, fabs((double)v[q] - ref));
          mx = fmax(mx, fabs(ref));
        }
      }
    }
    tc_release(ex, c);
    // block maxima (the operand tiles are free again)
    double* red = reinterpret_cast<double*>(c.tiles);
    red[ex.tid] = err;
    red[ex.nt + ex.tid] = mx;
    ex.sync();
    for (int s = ex.nt / 2; s > 0; s >>= 1) {
      if (ex.tid < s) {
        red[ex.tid] = fmax(red[ex.tid], red[ex.tid + s]);
        red[ex.nt + ex.tid] = fmax(red[ex.nt + ex.tid], red[ex.nt + ex.tid + s]);
      }
      ex.sync();
    }
    if (ex.tid == 0) {
      out[0] = red[0];
      out[1] = red[ex.nt];
      out[2] = ran ? 1.0 : 0.0;
    }
  }
};

// The bounded wait of the tensor-core kernels on an mbarrier that nothing
// arrives on: it must give up after `limit` polls and report it (status 4).
struct KWaitCheck {
  long long limit;
  int* status;
  __device__ void operator()(const KExec& ex, int) const {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ex.smem);
    if (ex.tid == 0)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(mbar)), "r"(1) : "memory");
    ex.sync();
    if (ex.tid == 0 && !tc_wait_bounded(tc_smem_addr(mbar), 0u, limit)) flag_error(status, 4);
    ex.sync();
  }
};

}  // namespace vb

using namespace vb;

extern "C" int vem_wait_selftest(long long limit) {
  if (limit < 0 || limit > (1ll << 30)) { set_last_error("vem_wait_selftest: limit out of range"); return VEM_EINVAL; }
  try {
    DBuf<int> status(1);
    status.zero();
    launch(KWaitCheck{limit, status.p}, 1, 32, 16, 0);
    VB_CUDA(cudaDeviceSynchronize());
    const auto st = status.download();
    if (st[0] == 4) {
      set_last_error("vem_wait_selftest: the bounded mbarrier wait gave up, as it must");
      return VEM_ETIMEOUT;
    }
    set_last_error("vem_wait_selftest: the wait on an mbarrier nobody arrives on completed");
    return VEM_ECUDA;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  }
}

extern "C" int vem_tc_selftest(double* max_err, double* max_ref) {
  if (!max_err || !max_ref) { set_last_error("vem_tc_selftest: null argument"); return VEM_EINVAL; }
  try {
    DBuf<double> out(3);
    DBuf<int> status(1);
    status.zero();
    out.zero();
    launch(KTcCheck{out.p, status.p}, 1, 256, TC_SMEM_BYTES, 0);
    VB_CUDA(cudaDeviceSynchronize());
    const auto h = out.download();
    const auto st = status.download();
    *max_err = h[0];
    *max_ref = h[1];
    if (st[0] != 0 || h[2] != 1.0) {
      set_last_error("vem_tc_selftest: the tensor-core product did not complete (bounded wait gave up)");
      return VEM_ETIMEOUT;
    }
    return VEM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  }
}

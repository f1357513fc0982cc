// Fifth-generation tensor cores (tcgen05) for the FP32 front factorization:
// the rank-32 trailing update of a dense front, C -= L (D L^T), in 128 x 128
// output tiles accumulated in tensor memory (TMEM).  FP32 operands are split
// into three TF32 parts, x = x0 + x1 + x2 (x0 = round(x), x1 = round(x - x0),
// x2 = x - x0 - x1, each exact in TF32), and each tile is the sum of the six
// products x_a y_b with a + b <= 2, accumulated in FP32: the dropped terms
// are of relative size 2^-33, so the update carries FP32 accuracy (a
// two-part split, 2^-22, was not enough for the local problems at a
// viscosity contrast of 1e4).
//
// Operand tiles are staged by the CTA's threads in shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix;
// core matrices adjacent along K 128 bytes apart, along M/N 1024 bytes
// apart for K = 32), one thread issues the 12 MMAs (K = 8 each) and commits
// them to an mbarrier, every wait on it is bounded, and the accumulator is
// read back with tcgen05.ld (warp w reads TMEM lanes 32 (w % 4) .. + 31).
#pragma once
#include "launch.h"

namespace vb {

constexpr int TC_M = 128, TC_N = 128, TC_K = 32;
constexpr int TC_TILE_FLOATS = TC_M * TC_K;   // one operand tile
constexpr int TC_PARTS = 3;                     // TF32 parts per operand
// shared memory of the TC path: A parts, B parts, then mbarrier + TMEM address
constexpr size_t TC_SMEM_BYTES = 2 * TC_PARTS * TC_TILE_FLOATS * sizeof(float) + 16;
// mbarrier polls before a wait gives up (about a second)
constexpr long long TC_WAIT_LIMIT = 1ll << 26;

struct TcCtx {
  float* tiles;        // [2*TC_PARTS][TC_TILE_FLOATS]: A parts 0..2, B parts 0..2
  uint64_t* mbar;
  uint32_t* taddr_slot;
  uint32_t taddr;
  uint32_t phase;
  int* status;         // set to 4 when a wait gives up
  bool failed;
};

__device__ inline uint32_t tc_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, descriptor version 1, no swizzle
__device__ inline uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// N = 128, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

// offset (in floats) of element (m, k) of a 128 x 32 operand tile
__device__ inline int tc_off(int m, int k) { return ((m >> 3) * 8 + (k >> 2)) * 32 + (m & 7) * 4 + (k & 3); }

__device__ inline float tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x into its three TF32 parts at offset o of the part tiles starting at t
__device__ inline void tc_split3(float x, float* t, int o) {
  const float x0 = tc_tf32(x);
  const float r = x - x0;
  const float x1 = tc_tf32(r);
  t[o] = x0;
  t[TC_TILE_FLOATS + o] = x1;
  t[2 * TC_TILE_FLOATS + o] = r - x1;
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation of 128 columns by warp 0, mbarrier set-up; all threads
__device__ inline void tc_init(const KExec& ex, TcCtx& c) {
  if ((ex.tid >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(c.taddr_slot)),
                 "r"(TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (ex.tid == 0)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(c.mbar)), "r"(1) : "memory");
  tc_fence_before();
  ex.sync();
  tc_fence_after();
  c.taddr = *c.taddr_slot;
  c.phase = 0;
  c.failed = false;
}

__device__ inline void tc_release(const KExec& ex, TcCtx& c) {
  tc_fence_before();
  ex.sync();
  tc_fence_after();
  if ((ex.tid >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.taddr), "r"(TC_N) : "memory");
}

__device__ inline bool tc_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}

__device__ inline void tc_mma(uint32_t taddr, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
      "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}

// 32 TMEM columns of this thread's lane into v
__device__ inline void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Polls the mbarrier phase at most `limit` times; false when it gave up.
__device__ inline bool tc_wait_bounded(uint32_t mbar, uint32_t phase, long long limit) {
  long long it = 0;
  bool done = false;
  while (!(done = tc_try_wait(mbar, phase)) && it < limit) ++it;
  return done;
}

// D = A B^T for the staged 128 x 32 tiles (A: rows of the output, B: its
// columns), split-TF32, into TMEM; thread 0 issues and waits (bounded), the
// outcome is shared through the CTA.  Returns false after a failed wait.
__device__ inline bool tc_product(const KExec& ex, TcCtx& c) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  ex.sync();
  tc_fence_after();
  __shared__ int tc_ok;
  if (ex.tid == 0) {
    const uint32_t base = tc_smem_addr(c.tiles);
    constexpr uint32_t TB = TC_TILE_FLOATS * 4;
    const uint32_t a0 = base, b0 = base + TC_PARTS * TB;
    // part pairs (a, b) with a + b <= 2, the small products first so that
    // they are summed before the large ones join the accumulator
    const int pa[6] = {1, 0, 2, 0, 1, 0}, pb[6] = {1, 2, 0, 1, 0, 0};
    // K = 8 per MMA: two core matrices (256 bytes) along K per step
    for (int q = 0; q < 6; ++q)
      for (int ks = 0; ks < TC_K / 8; ++ks) {
        const uint32_t o = ks * 256;
        tc_mma(c.taddr, tc_desc(a0 + pa[q] * TB + o, 128, 1024), tc_desc(b0 + pb[q] * TB + o, 128, 1024),
               (ks > 0 || q > 0) ? 1u : 0u);
      }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem_addr(c.mbar))
                 : "memory");
    const uint32_t mb = tc_smem_addr(c.mbar);
    bool done = tc_wait_bounded(mb, c.phase, TC_WAIT_LIMIT);
    if (!done) {
      // gave up: record it, wait once more (bounded) for the MMAs in flight
      flag_error(c.status, 4);
      done = tc_wait_bounded(mb, c.phase, TC_WAIT_LIMIT);
    }
    tc_ok = done ? 1 : 0;
  }
  tc_fence_before();
  ex.sync();
  tc_fence_after();
  c.phase ^= 1u;
  const bool ok = tc_ok != 0;
  if (!ok) c.failed = true;
  return ok;
}

}  // namespace vb

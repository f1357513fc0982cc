// Batched multifrontal LDL^T of the subdomain problems (nested-dissection
// trees, dense fronts, no pivoting: velocity pivots positive, pressure and
// multiplier pivots negative) and the triangular solves.  One CTA per front;
// all fronts of one tree height across all problems run in one launch.
//
// Front of node t: positions [p0, p0+np) (pivots) followed by its border
// (sorted positions eliminated by ancestors).  Storage: panel nf x np
// column-major (D on the diagonal, unit L below), update matrix nb x nb
// column-major (lower triangle valid), consumed by the parent.
#pragma once
#include "launch.h"
#include "bddc_dev.h"
#include "bddc_setup.h"
#include "tc.cuh"

#include <type_traits>

namespace vb {

VB_HD inline int front_index(const NodeDev& N, const int* bord, int x) {
  if (x < N.p0 + N.np) return x >= N.p0 ? x - N.p0 : -1;
  int lo = 0, hi = N.nb - 1;
  if (hi < 0) return -1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (bord[mid] < x) lo = mid + 1; else hi = mid;
  }
  return bord[lo] == x ? N.np + lo : -1;
}

// Trailing update of one panel (columns jb .. jb+nbk-1, rows and columns from
// c0 on, m of them) on the tensor cores: lower tiles (ti >= tk) of 128 x 128;
// each tile stages L (rows of the tile) and L D (its columns, once per tile
// column) as three TF32 parts, runs the split product into TMEM and
// subtracts it from the front
// (pivot columns in the panel, the rest in the update matrix).
// Front index -> deluxe entity group of a root-border DOF (-1: pivot or
// other border).  Only the diagonal entity blocks of the deluxe root update
// are used, and border DOFs are never pivots, so update entries between two
// different entities are never needed: trailing tiles lying entirely in
// such a block are skipped.  Border positions of a deluxe problem are
// grouped by entity in increasing position order.
struct FrontGroups {
  const int* bord;   // the front's border positions
  const int* pgrp;   // per problem position, or null (no deluxe problem)
  int np;
  VB_HD int of(int fi) const { return fi < np ? -1 : pgrp[bord[fi - np]]; }
  // lower tile rows [i0, ..), columns [k0, klast]: every pair in two different entities
  VB_HD bool cross(int i0, int k0, int klast) const {
    if (!pgrp || k0 < np) return false;
    const int gk = of(k0);
    return gk >= 0 && of(klast) < of(i0);
  }
};

__device__ inline bool tc_trailing_update(const KExec& ex, TcCtx& c, float* pan, float* upd, int np, int nb, int ld,
                                          int nf, int jb, int nbk, int c0, int m, const float* sd,
                                          const FrontGroups& fg) {
  float* A = c.tiles;                                // TF32 parts of the tile rows
  float* B = c.tiles + TC_PARTS * TC_TILE_FLOATS;    // TF32 parts of the tile columns
  const int nt = (m + TC_M - 1) / TC_M;
  const int w = ex.tid >> 5, lane = ex.tid & 31;
  const int rowblk = w & 3, colhalf = w >> 2;   // 8 warps: 4 lane groups x 2 column halves
  for (int tk = 0; tk < nt; ++tk) {
    const int k0 = c0 + tk * TC_N;
    // columns of the tile row: L D (scaled by the pivots), staged once per tk
    for (int q = ex.tid; q < TC_N * TC_K; q += ex.nt) {
      const int col = q / TC_N, mm = q % TC_N;
      const float y = (col < nbk && k0 + mm < nf) ? pan[(int64_t)(jb + col) * ld + k0 + mm] * sd[col] : 0.0f;
      tc_split3(y, B, tc_off(mm, col));
    }
    for (int ti = tk; ti < nt; ++ti) {
      const int i0 = c0 + ti * TC_M;
      if (fg.cross(i0, k0, min(k0 + TC_N, nf) - 1)) continue;
      for (int q = ex.tid; q < TC_M * TC_K; q += ex.nt) {
        const int col = q / TC_M, mm = q % TC_M;
        const float x = (col < nbk && i0 + mm < nf) ? pan[(int64_t)(jb + col) * ld + i0 + mm] : 0.0f;
        tc_split3(x, A, tc_off(mm, col));
      }
      if (!tc_product(ex, c)) return false;
      const int i = i0 + rowblk * 32 + lane;
      for (int cc = 0; cc < 2; ++cc) {
        float v[32];
        tc_ld32(c.taddr + ((uint32_t)(rowblk * 32) << 16) + (uint32_t)(colhalf * 64 + cc * 32), v);
        const int kb = k0 + colhalf * 64 + cc * 32;
        if (i < nf)
          for (int q = 0; q < 32; ++q) {
            const int k = kb + q;
            if (k >= nf || i < k) continue;
            if (k < np) pan[(int64_t)k * ld + i] -= v[q];
            else upd[(int64_t)(k - np) * nb + (i - np)] -= v[q];
          }
      }
      tc_fence_before();
      ex.sync();
      tc_fence_after();
    }
  }
  return true;
}

// barrier of one group of 256 threads (named barrier 1 + grp), or of the
// whole CTA when it works as a single group
VB_HD inline void group_sync(const KExec& ex, int ngrp, int grp) {
#ifdef __CUDA_ARCH__
  if (ngrp > 1) {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(256) : "memory");
    return;
  }
#endif
  (void)grp;
  ex.sync();
}

// One 64 x 64 tile (rows i0.., columns k0..) of the trailing update of a
// front by the pivot columns [ka, kb) (unit L below the diagonal, D on it;
// sdv[c - dbase] = D of column c), by a group of 256 threads (gt, gnt: index
// and size in the group, 4 x 4 outputs per thread accumulated in registers
// over the whole K range, which streams through shared memory 32 columns at
// a time):  C[i][k] -= sum_c L[i][c] D[c] L[k][c]  for i >= k, k < ce (pivot
// columns in the panel, the rest in the update matrix).
template <class T>
VB_HD inline void trailing_tile(const KExec& ex, T* pan, T* upd, int np, int nb, int ld, int ka, int kb, int i0,
                                int k0, int ce, const T* sdv, int dbase, T* sL, T* sR, int ngrp, int grp, int gt,
                                int gnt, bool act) {
  constexpr int NBK = 32, TT = 64;
  const int nf = np + nb;
  T acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  const int tr = gt % 16, tcl = gt / 16;
  for (int kc = ka; kc < kb; kc += NBK) {
    const int nkc = kb - kc < NBK ? kb - kc : NBK;
    if (act)
      for (int q = gt; q < TT * NBK; q += gnt) {
        const int r = q % TT, c = q / TT;
        sL[q] = (c < nkc && i0 + r < nf) ? pan[(int64_t)(kc + c) * ld + i0 + r] : (T)0;
        sR[q] = (c < nkc && k0 + r < nf) ? pan[(int64_t)(kc + c) * ld + k0 + r] * sdv[kc + c - dbase] : (T)0;
      }
    group_sync(ex, ngrp, grp);
    if (act && gt < 256)
      for (int c = 0; c < nkc; ++c) {
        T li[4], rk[4];
        for (int a = 0; a < 4; ++a) li[a] = sL[c * TT + tr + 16 * a];
        for (int bb = 0; bb < 4; ++bb) rk[bb] = sR[c * TT + tcl + 16 * bb];
        for (int a = 0; a < 4; ++a)
          for (int bb = 0; bb < 4; ++bb) acc[a][bb] += li[a] * rk[bb];
      }
    group_sync(ex, ngrp, grp);
  }
  if (act && gt < 256)
    for (int bb = 0; bb < 4; ++bb) {
      const int k = k0 + tcl + 16 * bb;
      if (k >= nf || k >= ce) continue;
      for (int a = 0; a < 4; ++a) {
        const int i = i0 + tr + 16 * a;
        if (i >= nf || i < k) continue;
        if (k < np) pan[(int64_t)k * ld + i] -= acc[a][bb];
        else upd[(int64_t)(k - np) * nb + (i - np)] -= acc[a][bb];
      }
    }
}

// Trailing update of a front by the pivot columns [ka, kb) for rows in
// [r0, nf) and columns in [r0, ce): every lower 64 x 64 tile, one per group
// of 256 threads; tiles lying between two different deluxe entities are
// skipped.
template <class T>
VB_HD inline void front_trailing(const KExec& ex, T* pan, T* upd, int np, int nb, int ld, int ka, int kb, int r0,
                                 int ce, const T* sdv, int dbase, T* sL, T* sR, int ngrp, int grp, int gt, int gnt,
                                 const FrontGroups& fg) {
  constexpr int TT = 64;
  const int nf = np + nb;
  if (r0 >= nf || r0 >= ce || ka >= kb) return;
  const int nrt = (nf - r0 + TT - 1) / TT, nct = (ce - r0 + TT - 1) / TT;
  const int ntot = nct * nrt - nct * (nct - 1) / 2;   // lower tiles, tk-major
  const int rounds = (ntot + ngrp - 1) / ngrp;
  for (int rr = 0; rr < rounds; ++rr) {
    const int tt = rr * ngrp + grp;
    bool act = tt < ntot;
    int tk = 0, ti = 0;
    if (act) {
      int rem = tt;
      while (rem >= nrt - tk) { rem -= nrt - tk; ++tk; }
      ti = tk + rem;
    }
    const int k0 = r0 + tk * TT, i0 = r0 + ti * TT;
    if (act && fg.cross(i0, k0, (k0 + TT < nf ? k0 + TT : nf) - 1)) act = false;
    trailing_tile<T>(ex, pan, upd, np, nb, ld, ka, kb, i0, k0, ce, sdv, dbase, sL, sR, ngrp, grp, gt, gnt, act);
  }
}

// Columns [jb, jb + nbk) of a front, one by one: pivot sign check, rank-1
// update of the rest of the block, scaling by the pivot.
template <class T>
VB_HD inline void front_columns(const KExec& ex, T* pan, int nf, int ld, const int* piv_type, int* status, int jb,
                                int nbk) {
  for (int jj = 0; jj < nbk; ++jj) {
    const int j = jb + jj;
    T* cj = pan + (int64_t)j * ld;
    const T dj = cj[j];
    if (ex.tid == 0) {
      const double sgn = (!piv_type || piv_type[j] == DT_VEL) ? 1.0 : -1.0;
      if (!((double)dj * sgn > 0.0)) flag_error(status, 3);
    }
    const T inv = (T)1 / dj;
    const int nk = jb + nbk - j - 1, nr = nf - j - 1;
    for (int64_t idx = ex.tid; idx < (int64_t)nk * nr; idx += ex.nt) {
      const int kk = j + 1 + (int)(idx / nr), ii = j + 1 + (int)(idx % nr);
      if (ii < kk) continue;
      pan[(int64_t)kk * ld + ii] -= cj[ii] * cj[kk] * inv;
    }
    ex.sync();
    for (int i = j + 1 + ex.tid; i < nf; i += ex.nt) cj[i] *= inv;
    ex.sync();
  }
}

// selective inversion: overwrite the unit lower L11 by L11^{-1} (unit
// lower), column by column from the right, so that the triangular sweeps
// become matrix-vector products over independent rows/columns
template <class T>
VB_HD inline void front_invert(const KExec& ex, T* pan, int np, int ld) {
  T* tmp = reinterpret_cast<T*>(ex.smem);
  for (int j = np - 2; j >= 0; --j) {
    for (int k = j + 1 + ex.tid; k < np; k += ex.nt) tmp[k] = pan[(int64_t)j * ld + k];
    ex.sync();
    for (int i = j + 1 + ex.tid; i < np; i += ex.nt) {
      T acc = tmp[i];
      for (int k = j + 1; k < i; ++k) acc += pan[(int64_t)k * ld + i] * tmp[k];
      pan[(int64_t)j * ld + i] = -acc;
    }
    ex.sync();
  }
}

// Shared-memory layout of the factorization of one front: per group of 256
// threads two 64 x 32 operand tiles, then the NBO diagonal entries of the
// current outer panel.
template <class T>
struct FrontSmem {
  static constexpr int NBK = 32, TT = 64, NBO = 128;
  T *sL, *sR, *sd;
  int ngrp, grp, gt, gnt;
  VB_HD explicit FrontSmem(const KExec& ex) {
    ngrp = ex.nt >= 512 ? ex.nt / 256 : 1;
    grp = ngrp > 1 ? ex.tid / 256 : 0;
    gt = ngrp > 1 ? ex.tid % 256 : ex.tid;
    gnt = ngrp > 1 ? 256 : ex.nt;
    sL = reinterpret_cast<T*>(ex.smem) + (int64_t)grp * 2 * TT * NBK;
    sR = sL + TT * NBK;
    sd = reinterpret_cast<T*>(ex.smem) + (int64_t)ngrp * 2 * TT * NBK;
  }
};

// Outer panel [JB, JE) of a front on the FMA units: inner blocks of NBK
// columns, each factored column by column and followed by the rank-NBK
// update of the rest of the outer panel; leaves the panel's D in sm.sd.
template <class T>
VB_HD inline void front_panel(const KExec& ex, const FrontSmem<T>& sm, T* pan, T* upd, int np, int nb, int ld,
                              const int* piv_type, int* status, int JB, int JE, const FrontGroups& fg) {
  const int nf = np + nb;
  for (int jb = JB; jb < JE; jb += FrontSmem<T>::NBK) {
    const int nbk = JE - jb < FrontSmem<T>::NBK ? JE - jb : FrontSmem<T>::NBK;
    front_columns<T>(ex, pan, nf, ld, piv_type, status, jb, nbk);
    for (int jj = ex.tid; jj < nbk; jj += ex.nt) sm.sd[jb - JB + jj] = pan[(int64_t)(jb + jj) * ld + jb + jj];
    ex.sync();
    const int c0 = jb + nbk;
    front_trailing<T>(ex, pan, upd, np, nb, ld, jb, c0, c0, JE, sm.sd, JB, sm.sL, sm.sR, sm.ngrp, sm.grp, sm.gt,
                      sm.gnt, fg);
    ex.sync();
  }
}

// Blocked right-looking partial LDL^T of one dense front (panel nf x np and
// update block nb x nb, column-major, lower triangles), followed by the
// in-place inversion of the unit lower diagonal block L11.  piv_type (may be
// null: all positive) gives the expected pivot sign per pivot (velocity
// positive; pressure and multiplier negative); a violation sets status 3.
// Two levels of blocking: outer panels of NBO pivot columns, factored as
// inner blocks of NBK columns (column by column, then a rank-NBK update of
// the rest of the outer panel), then one rank-NBO update of the trailing
// front, so that the trailing front is read and written once per NBO
// columns.  With more than 256 threads the CTA works as groups of 256, each
// on its own trailing tile (named barriers per group).  With the tensor
// cores (tc) the trailing update runs after every NBK columns instead.
// want_update = false: the update matrix (border x border block) is not
// needed by the caller and is not computed (the border rows of the panel,
// L21, are).
template <class T>
VB_HD inline void front_ldlt(const KExec& ex, T* pan, T* upd, int np, int nb, int ld, const int* piv_type,
                             int* status, TcCtx* tc = nullptr, FrontGroups fg = FrontGroups{nullptr, nullptr, 0},
                             bool want_update = true) {
  const int nf = np + nb;
  const int ce_all = want_update ? nf : np;
  const FrontSmem<T> sm(ex);
  constexpr int NBK = FrontSmem<T>::NBK, TT = FrontSmem<T>::TT, NBO = FrontSmem<T>::NBO;
  if (!tc) {
    for (int JB = 0; JB < np; JB += NBO) {
      const int JE = np - JB < NBO ? np : JB + NBO;
      front_panel<T>(ex, sm, pan, upd, np, nb, ld, piv_type, status, JB, JE, fg);
      // rank-(JE - JB) update of the trailing front
      front_trailing<T>(ex, pan, upd, np, nb, ld, JB, JE, JE, ce_all, sm.sd, JB, sm.sL, sm.sR, sm.ngrp, sm.grp,
                        sm.gt, sm.gnt, fg);
      ex.sync();
    }
  } else {
    for (int jb = 0; jb < np; jb += NBK) {
      const int nbk = np - jb < NBK ? np - jb : NBK;
      front_columns<T>(ex, pan, nf, ld, piv_type, status, jb, nbk);
      for (int jj = ex.tid; jj < nbk; jj += ex.nt) sm.sd[jj] = pan[(int64_t)(jb + jj) * ld + jb + jj];
      ex.sync();
      const int c0 = jb + nbk, m = nf - c0;
      if (m <= 0) continue;
#ifdef __CUDA_ARCH__
      if constexpr (std::is_same<T, float>::value) {
        if (m > TT) {
          // tensor-core tiles (split TF32, 128 x 128, accumulators in TMEM)
          if (!tc_trailing_update(ex, *tc, pan, upd, np, nb, ld, nf, jb, nbk, c0, m, sm.sd, fg)) return;
          continue;
        }
      }
#endif
      front_trailing<T>(ex, pan, upd, np, nb, ld, jb, c0, c0, ce_all, sm.sd, jb, sm.sL, sm.sR, sm.ngrp, sm.grp,
                        sm.gt, sm.gnt, fg);
      ex.sync();
    }
  }
  front_invert<T>(ex, pan, np, ld);
}

template <class T, bool UseTC = false>
struct KFactor {
  BddcView V;
  const int* list;
  T* F;
  T* U;
  int* status;
  size_t tc_smem_off = 0;   // UseTC: byte offset of the tensor-core tiles in shared memory
  // mode 0: the whole front; the split form of a level with few large
  // fronts: 1 assembly only, 2 the outer panel [JB, JB + NBO) (its trailing
  // update is KFactorTiles), 3 the inversion of L11 only
  int mode = 0, JB = 0;
  __device__ void operator()(const KExec& ex, int blk) const {
    if (mode != 0) {
      split_step(ex, blk);
      return;
    }
    if constexpr (UseTC) {
      TcCtx c;
      c.tiles = reinterpret_cast<float*>(reinterpret_cast<char*>(ex.smem) + tc_smem_off);
      c.mbar = reinterpret_cast<uint64_t*>(c.tiles + 2 * TC_PARTS * TC_TILE_FLOATS);
      c.taddr_slot = reinterpret_cast<uint32_t*>(c.mbar + 1);
      c.status = status;
      tc_init(ex, c);
      body(ex, blk, &c);
      tc_release(ex, c);
      return;
    }
    body(ex, blk, nullptr);
  }
  __device__ void split_step(const KExec& ex, int blk) const {
    const int t = list[blk];
    const NodeDev N = V.nodes[t];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nb = N.nb, ld = N.ld;
    T* pan = F + N.panel_off;
    T* upd = U + N.upd_off;
    if (mode == 1) {
      assemble(ex, blk);
    } else if (mode == 2) {
      if (JB >= np) return;
      const int JE = np - JB < FrontSmem<T>::NBO ? np : JB + FrontSmem<T>::NBO;
      const FrontSmem<T> sm(ex);
      const FrontGroups fg{V.border + N.border_off, P.kind == PK_DELUXE ? V.bgrp + P.pos_off : nullptr, np};
      front_panel<T>(ex, sm, pan, upd, np, nb, ld, V.dtype + P.pos_off + N.p0, status, JB, JE, fg);
    } else {
      front_invert<T>(ex, pan, np, ld);
    }
  }
  __device__ void body(const KExec& ex, int blk, TcCtx* tc) const {
    assemble(ex, blk);
    const int t = list[blk];
    const NodeDev N = V.nodes[t];
    const ProbDev P = V.probs[N.prob];
    const FrontGroups fg{V.border + N.border_off, P.kind == PK_DELUXE ? V.bgrp + P.pos_off : nullptr, N.np};
    front_ldlt<T>(ex, F + N.panel_off, U + N.upd_off, N.np, N.nb, N.ld, V.dtype + P.pos_off + N.p0, status, tc, fg);
  }
  // zero the front, add the original matrix entries of its pivot columns
  // and the children's update matrices
  __device__ void assemble(const KExec& ex, int blk) const {
    const int t = list[blk];
    const NodeDev N = V.nodes[t];
    const ProbDev P = V.probs[N.prob];
    const SubDev S = V.subs[P.sub];
    const int np = N.np, nb = N.nb, ld = N.ld;
    const int npk = V.np;
    T* pan = F + N.panel_off;
    T* upd = U + N.upd_off;
    const int* bord = V.border + N.border_off;
    for (int64_t i = ex.tid; i < (int64_t)ld * np; i += ex.nt) pan[i] = (T)0;
    for (int64_t i = ex.tid; i < (int64_t)nb * nb; i += ex.nt) upd[i] = (T)0;
    ex.sync();
    // original matrix entries of the pivot columns (one thread per column)
    for (int j = ex.tid; j < np; j += ex.nt) {
      const int pos = N.p0 + j;
      const int dt = V.dtype[P.pos_off + pos];
      const int src = V.dsrc[P.pos_off + pos];
      T* colp = pan + (int64_t)j * ld;
      if (dt == DT_VEL) {
        const int* vp = V.vadj_ptr + S.vadj_ptr_off;
        for (int q = vp[src]; q < vp[src + 1]; ++q) {
          const int le = V.vadj[S.vadj_off + 2 * q], a = V.vadj[S.vadj_off + 2 * q + 1];
          const int e = V.sub_elems[S.elem_off + le];
          const int nK = (int)(V.offK[e + 1] - V.offK[e]);
          const int* ep = V.elpos + P.elpos_off + V.elptr[P.elptr_off + le];
          const double* Ae = V.A + V.offK2[e];
          const double* Be = V.B + (int64_t)npk * V.offK[e];
          for (int b = 0; b < nK + npk; ++b) {
            const int x = ep[b];
            if (x < pos) continue;
            const double v = b < nK ? Ae[(int64_t)a * nK + b] : Be[(int64_t)(b - nK) * nK + a];
            const int fi = front_index(N, bord, x);
            if (fi < 0) { flag_error(status, 2); continue; }
            colp[fi] += (T)v;
          }
        }
        if (P.kind == PK_NEUMANN) {
          const int* cp = V.vcon_ptr + S.vcon_ptr_off;
          for (int q = cp[src]; q < cp[src + 1]; ++q) {
            const int x = P.mult0 + V.vcon_id[S.vcon_off + q];
            const int fi = front_index(N, bord, x);
            if (fi < 0) { flag_error(status, 2); continue; }
            colp[fi] += (T)V.vcon_coef[S.vcon_off + q];
          }
        }
      } else if (dt == DT_PRESS) {
        const int le = src / npk, a = src % npk;
        const int e = V.sub_elems[S.elem_off + le];
        const int nK = (int)(V.offK[e + 1] - V.offK[e]);
        const int* ep = V.elpos + P.elpos_off + V.elptr[P.elptr_off + le];
        const double* Be = V.B + (int64_t)npk * V.offK[e];
        for (int b = 0; b < nK; ++b) {
          const int x = ep[b];
          if (x < pos) continue;
          const int fi = front_index(N, bord, x);
          if (fi < 0) { flag_error(status, 2); continue; }
          colp[fi] += (T)Be[(int64_t)a * nK + b];
        }
      }
    }
    // deluxe root: entries between border-only DOFs (the face block K_FF)
    if (N.flags & 1) {
      for (int i = ex.tid; i < nb; i += ex.nt) {
        const int x = bord[i];
        const int v = V.dsrc[P.pos_off + x];
        const int* vp = V.vadj_ptr + S.vadj_ptr_off;
        for (int q = vp[v]; q < vp[v + 1]; ++q) {
          const int le = V.vadj[S.vadj_off + 2 * q], a = V.vadj[S.vadj_off + 2 * q + 1];
          const int e = V.sub_elems[S.elem_off + le];
          const int nK = (int)(V.offK[e + 1] - V.offK[e]);
          const int* ep = V.elpos + P.elpos_off + V.elptr[P.elptr_off + le];
          const double* Ae = V.A + V.offK2[e];
          for (int b = 0; b < nK; ++b) {
            const int y = ep[b];
            if (y < P.npiv || y > x) continue;
            const int fk = front_index(N, bord, y);
            if (fk < np) { flag_error(status, 2); continue; }
            upd[(int64_t)(fk - np) * nb + i] += (T)Ae[(int64_t)a * nK + b];
          }
        }
      }
    }
    ex.sync();
    // extend-add of the children's update matrices
    for (int c = 0; c < N.nchild; ++c) {
      const NodeDev C = V.nodes[V.children[N.first_child + c]];
      const int* rel = V.rel + C.rel_off;
      const T* Uc = U + C.upd_off;
      const int nbc = C.nb;
      for (int64_t idx = ex.tid; idx < (int64_t)nbc * nbc; idx += ex.nt) {
        const int kk = (int)(idx / nbc), ii = (int)(idx % nbc);
        if (ii < kk) continue;
        const int rc = rel[kk], rr = rel[ii];
        const T v = Uc[idx];
        if (rc < np) pan[(int64_t)rc * ld + rr] += v;
        else upd[(int64_t)(rc - np) * nb + (rr - np)] += v;
      }
      ex.sync();
    }
    (void)bord;
  }
};

// The trailing update of the split form: one 64 x 64 tile per CTA of 256
// threads, of one front of the level, by the pivot columns [JB, JE) of its
// current outer panel (D read from the panel's diagonal).
struct FrontTile {
  int node, i0, k0;
};
template <class T>
struct KFactorTiles {
  BddcView V;
  const FrontTile* tiles;
  T* F;
  T* U;
  int JB;
  __device__ void operator()(const KExec& ex, int blk) const {
    const FrontTile tl = tiles[blk];
    const NodeDev N = V.nodes[tl.node];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nb = N.nb, nf = np + nb, ld = N.ld;
    const int JE = np - JB < FrontSmem<T>::NBO ? np : JB + FrontSmem<T>::NBO;
    const FrontGroups fg{V.border + N.border_off, P.kind == PK_DELUXE ? V.bgrp + P.pos_off : nullptr, np};
    if (fg.cross(tl.i0, tl.k0, (tl.k0 + 64 < nf ? tl.k0 + 64 : nf) - 1)) return;
    T* pan = F + N.panel_off;
    T* sL = reinterpret_cast<T*>(ex.smem);
    T* sR = sL + 64 * 32;
    T* sd = sR + 64 * 32;
    for (int c = ex.tid; c < JE - JB; c += ex.nt) sd[c] = pan[(int64_t)(JB + c) * ld + JB + c];
    ex.sync();
    trailing_tile<T>(ex, pan, U + N.upd_off, np, nb, ld, JB, JE, tl.i0, tl.k0, nf, sd, JB, sL, sR, 1, 0, ex.tid,
                     ex.nt, true);
  }
};

// sum over the 32 lanes of a warp
VB_HD inline double warp_sum(double v) {
#ifdef __CUDA_ARCH__
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
  return v;
}
VB_HD inline float warp_sum(float v) {
#ifdef __CUDA_ARCH__
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
  return v;
}

// Triangular sweeps over one tree level, split into tasks of up to TASK
// rows (or columns) of one front, so that large fronts spread over many CTAs.
// A task record: node id, first row/column, count.
struct SolveTask {
  int node, start, count;
};
constexpr int TASK = 128;
constexpr int BCOLS = 32;   // pivot columns per backward-sweep task (4 per warp)

// The vectors of a sweep (right-hand sides and solutions X, front vectors
// FV, update vectors UV) are held in the factor's precision T.

// forward (1): front vector of each node = its own right-hand side entries
// plus the children's update vectors (extend-add), one CTA per node
template <class T>
struct KFwdGather {
  BddcView V;
  const int* list;
  const T* X;    // [vec_off*nrhs + r*n + pos]
  const T* UV;   // [uvec_off*nrhs + r*nb + i]
  T* FV;         // [fv_off*nrhs + r*nf + i]
  const int64_t* fv_off;
  int nrhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int t = list[blk];
    const NodeDev N = V.nodes[t];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nf = N.np + N.nb;
    for (int r = 0; r < nrhs; ++r) {
      const T* x = X + P.vec_off * nrhs + (int64_t)r * P.n;
      T* f = FV + fv_off[t] * nrhs + (int64_t)r * nf;
      for (int i = ex.tid; i < nf; i += ex.nt) f[i] = i < np ? x[N.p0 + i] : (T)0;
      ex.sync();
      for (int c = 0; c < N.nchild; ++c) {
        const NodeDev C = V.nodes[V.children[N.first_child + c]];
        const int* rel = V.rel + C.rel_off;
        const T* uc = UV + C.uvec_off * nrhs + (int64_t)r * C.nb;
        for (int i = ex.tid; i < C.nb; i += ex.nt) f[rel[i]] += uc[i];
        ex.sync();
      }
    }
  }
};

// Right-hand sides are processed in groups of RB (template argument): every
// factor entry read from memory serves RB accumulators (RB = 1 for the
// single right-hand side of the CG iteration, 4 for the coarse basis).

// 16-byte vector loads of factor columns: W consecutive rows per load (the
// panels are 4-element aligned with a leading dimension divisible by 4)
template <class T>
struct VecW;
template <>
struct VecW<double> {
  static constexpr int W = 2;
};
template <>
struct VecW<float> {
  static constexpr int W = 4;
};
VB_HD inline void vload(const double* p, double* o) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x;
  o[1] = v.y;
}
VB_HD inline void vload(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}

// The sweeps accumulate and store in the factor's precision: FP64 arithmetic
// (conversions included) runs at a small fraction of the FP32 rate on this
// GPU, and an FP32-local solve is followed by refinement with an FP64
// residual anyway.

// Forward tasks cover up to FVEC W-row vectors (one per lane); the warps of
// the CTA split the column range and their partial sums are added in a
// fixed order through shared memory.  Loads are issued in groups of 4
// columns so that each lane keeps several 16-byte loads in flight.
constexpr int FVEC = 32;
constexpr int FWARPS = 8;
// backward tasks: each warp takes BCOL adjacent columns at a time
constexpr int BCOL = 4;

// rows [i0, i0+W) of L[.][k] * x_k accumulated for k in [ka, kb); entries
// with row <= k (diagonal block of the unit lower inverse) skipped when
// `tri` is set
template <class T, int RB>
VB_HD inline void fwd_accum(const T* base, int ld, const T* xs, int xld, int ka, int kb, int i0, bool tri,
                            T (*acc)[RB]) {
  constexpr int W = VecW<T>::W;
  const int kfull = tri ? (kb < i0 ? kb : i0) : kb;
  int k = ka;
  for (; k + 4 <= kfull; k += 4) {
    T v0[W], v1[W], v2[W], v3[W];
    vload(base + (int64_t)k * ld, v0);
    vload(base + (int64_t)(k + 1) * ld, v1);
    vload(base + (int64_t)(k + 2) * ld, v2);
    vload(base + (int64_t)(k + 3) * ld, v3);
    for (int r = 0; r < RB; ++r) {
      const T* x = xs + r * xld + k;
      for (int j = 0; j < W; ++j) acc[j][r] += v0[j] * x[0] + v1[j] * x[1] + v2[j] * x[2] + v3[j] * x[3];
    }
  }
  for (; k < kfull; ++k) {
    T v[W];
    vload(base + (int64_t)k * ld, v);
    for (int r = 0; r < RB; ++r)
      for (int j = 0; j < W; ++j) acc[j][r] += v[j] * xs[r * xld + k];
  }
  if (!tri) return;
  const int kt = kb < i0 + W - 1 ? kb : i0 + W - 1;
  for (k = ka > i0 ? ka : i0; k < kt; ++k) {
    T v[W];
    vload(base + (int64_t)k * ld, v);
    for (int r = 0; r < RB; ++r)
      for (int j = 0; j < W; ++j)
        if (i0 + j > k) acc[j][r] += v[j] * xs[r * xld + k];
  }
}

// forward (2): y_p = L11^{-1} f_p (L11^{-1} unit lower, stored in place);
// a task is up to FVEC W-row vectors of the pivot rows
template <class T, int RB>
struct KFwdPivots {
  BddcView V;
  const SolveTask* tasks;   // {node, first vector, vectors}
  const T* F;
  const T* FV;
  const int64_t* fv_off;
  T* X;
  int nrhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    constexpr int W = VecW<T>::W;
    const SolveTask tk = tasks[blk];
    const NodeDev N = V.nodes[tk.node];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nf = N.np + N.nb, ld = N.ld;
    const T* pan = F + N.panel_off;
    const int rend = W * (tk.start + tk.count);
    const int kmax = rend < np ? rend : np;
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    const int kc = (kmax + nw - 1) / nw, ka = w * kc, kb = ka + kc < kmax ? ka + kc : kmax;
    T* fs = reinterpret_cast<T*>(ex.smem);        // [RB][kmax]
    T* red = fs + ((RB * kmax + 3) & ~3);         // [nw][FVEC][W][RB]
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
      for (int q = ex.tid; q < RB * kmax; q += ex.nt) {
        const int r = q / kmax, k = q % kmax;
        fs[q] = r < nr ? FV[fv_off[tk.node] * nrhs + (int64_t)(r0 + r) * nf + k] : (T)0;
      }
      ex.sync();
      for (int v = lane; v < tk.count; v += ws) {
        const int i0 = W * (tk.start + v);
        T acc[W][RB];
        for (int j = 0; j < W; ++j)
          for (int r = 0; r < RB; ++r) acc[j][r] = (T)0;
        fwd_accum<T, RB>(pan + i0, ld, fs, kmax, ka, kb, i0, true, acc);
        for (int j = 0; j < W; ++j)
          for (int r = 0; r < RB; ++r) red[((w * FVEC + v) * W + j) * RB + r] = acc[j][r];
      }
      ex.sync();
      for (int q = ex.tid; q < tk.count * W; q += ex.nt) {
        const int v = q / W, j = q % W, row = W * (tk.start + v) + j;
        if (row >= np) continue;
        for (int r = 0; r < nr; ++r) {
          T y = fs[r * kmax + row];
          for (int u = 0; u < nw; ++u) y += red[((u * FVEC + v) * W + j) * RB + r];
          X[P.vec_off * nrhs + (int64_t)(r0 + r) * P.n + N.p0 + row] = y;
        }
      }
      ex.sync();
    }
  }
};

// forward (3): update vector u = f_b - L21 y; a task is up to FVEC W-row
// vectors of the border rows (aligned base floor(np/W)*W)
template <class T, int RB>
struct KFwdBorder {
  BddcView V;
  const SolveTask* tasks;
  const T* F;
  const T* FV;
  const int64_t* fv_off;
  const T* X;
  T* UV;
  int nrhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    constexpr int W = VecW<T>::W;
    const SolveTask tk = tasks[blk];
    const NodeDev N = V.nodes[tk.node];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nf = N.np + N.nb, ld = N.ld;
    const int a0 = (np / W) * W;
    const T* pan = F + N.panel_off;
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    const int kc = (np + nw - 1) / nw, ka = w * kc, kb = ka + kc < np ? ka + kc : np;
    T* ys = reinterpret_cast<T*>(ex.smem);      // [RB][np]
    T* red = ys + ((RB * np + 3) & ~3);         // [nw][FVEC][W][RB]
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
      for (int q = ex.tid; q < RB * np; q += ex.nt) {
        const int r = q / np, k = q % np;
        ys[q] = r < nr ? X[P.vec_off * nrhs + (int64_t)(r0 + r) * P.n + N.p0 + k] : (T)0;
      }
      ex.sync();
      for (int v = lane; v < tk.count; v += ws) {
        const int i0 = a0 + W * (tk.start + v);
        T acc[W][RB];
        for (int j = 0; j < W; ++j)
          for (int r = 0; r < RB; ++r) acc[j][r] = (T)0;
        fwd_accum<T, RB>(pan + i0, ld, ys, np, ka, kb, i0, false, acc);
        for (int j = 0; j < W; ++j)
          for (int r = 0; r < RB; ++r) red[((w * FVEC + v) * W + j) * RB + r] = acc[j][r];
      }
      ex.sync();
      for (int q = ex.tid; q < tk.count * W; q += ex.nt) {
        const int v = q / W, j = q % W, row = a0 + W * (tk.start + v) + j;
        if (row < np || row >= nf) continue;
        for (int r = 0; r < nr; ++r) {
          T s = (T)0;
          for (int u = 0; u < nw; ++u) s += red[((u * FVEC + v) * W + j) * RB + r];
          const T* f = FV + fv_off[tk.node] * nrhs + (int64_t)(r0 + r) * nf;
          UV[N.uvec_off * nrhs + (int64_t)(r0 + r) * N.nb + (row - np)] = f[row] - s;
        }
      }
      ex.sync();
    }
  }
};

// sum over rows [lo, hi) of column segment c (vectors from aligned row b0)
// of c[row] * xs[r*xld + row - xoff], lanes striding over W-row vectors
template <class T, int RB>
VB_HD inline void col_dot(const T* c, int b0, int lo, int hi, const T* xs, int xld, int xoff, int lane, int ws,
                          T* acc) {
  constexpr int W = VecW<T>::W;
  const int nvec = hi > b0 ? (hi - b0 + W - 1) / W : 0;
  int q = lane;
  for (; q + 3 * ws < nvec; q += 4 * ws) {
    T v[4][W];
    for (int u = 0; u < 4; ++u) vload(c + W * (q + u * ws), v[u]);
    for (int u = 0; u < 4; ++u)
      for (int jj = 0; jj < W; ++jj) {
        const int row = b0 + W * (q + u * ws) + jj;
        if (row < lo || row >= hi) continue;
        for (int r = 0; r < RB; ++r) acc[r] += v[u][jj] * xs[r * xld + row - xoff];
      }
  }
  for (; q < nvec; q += ws) {
    T v[W];
    vload(c + W * q, v);
    for (int jj = 0; jj < W; ++jj) {
      const int row = b0 + W * q + jj;
      if (row < lo || row >= hi) continue;
      for (int r = 0; r < RB; ++r) acc[r] += v[jj] * xs[r * xld + row - xoff];
    }
  }
}

// NC adjacent columns at once (column u at c + u*ld, u < ncol): per column
// the sum over rows [lo[u], hi) of c_u[row] * x[row], lanes striding over
// W-row vectors from the aligned row b0.  x is staged in shared memory from
// row b0 on (xs[r*xld + row - b0], zero past hi), so each factor vector meets
// one aligned shared-memory vector load per right-hand side; rows below
// lo[u] are masked only in the vectors that reach below lo_max = max lo[u].
template <class T, int RB, int NC>
__device__ inline void col_dot_n(const T* c, int64_t ld, int ncol, int b0, int lo_max, const int* lo, int hi,
                                 const T* xs, int xld, int lane, T (*acc)[RB]) {
  constexpr int W = VecW<T>::W;
  const int nvec = hi > b0 ? (hi - b0 + W - 1) / W : 0;
#pragma unroll 2
  for (int q = lane; q < nvec; q += 32) {
    T v[NC][W];
#pragma unroll
    for (int u = 0; u < NC; ++u)
      if (u < ncol) vload(c + u * ld + W * q, v[u]);
    T xv[RB][W];
#pragma unroll
    for (int r = 0; r < RB; ++r) vload(xs + r * xld + W * q, xv[r]);
    const int rb = b0 + W * q;
    if (rb < lo_max) {
#pragma unroll
      for (int u = 0; u < NC; ++u)
#pragma unroll
        for (int jj = 0; jj < W; ++jj)
          if (u < ncol && rb + jj >= lo[u])
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[u][r] += v[u][jj] * xv[r][jj];
    } else {
#pragma unroll
      for (int u = 0; u < NC; ++u)
        if (u < ncol)
#pragma unroll
          for (int jj = 0; jj < W; ++jj)
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[u][r] += v[u][jj] * xv[r][jj];
    }
  }
}

// backward (1): t_j = y_j / d_j - sum_border L21[i][j] x_i for a task of
// pivot columns (one warp per column, lanes along W-row vectors)
template <class T, int RB>
struct KBwdBorder {
  BddcView V;
  const SolveTask* tasks;
  const T* F;
  const T* X;
  T* TV;             // [fv_off*nrhs + r*nf + j] (reuses the front-vector store)
  const int64_t* fv_off;
  int nrhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    constexpr int W = VecW<T>::W;
    const SolveTask tk = tasks[blk];
    const NodeDev N = V.nodes[tk.node];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nb = N.nb, nf = np + nb, ld = N.ld;
    const int a0 = (np / W) * W;
    const T* pan = F + N.panel_off;
    const int* bord = V.border + N.border_off;
    // border values staged from the aligned row a0: xb[r*xld + row - a0],
    // zero for the pivot rows below np and past nf
    const int xld = ((nf - a0 + W - 1) / W) * W;
    T* xb = reinterpret_cast<T*>(ex.smem);   // [RB][xld]
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
      for (int q = ex.tid; q < RB * xld; q += ex.nt) {
        const int r = q / xld, row = a0 + q % xld;
        xb[q] = (r < nr && row >= np && row < nf)
                    ? X[P.vec_off * nrhs + (int64_t)(r0 + r) * P.n + bord[row - np]] : (T)0;
      }
      ex.sync();
      const int jend = tk.start + tk.count;
      for (int j0 = tk.start + BCOL * w; j0 < jend; j0 += BCOL * nw) {
        const int ncol = jend - j0 < BCOL ? jend - j0 : BCOL;
        T acc[BCOL][RB];
        int lo[BCOL];
        for (int u = 0; u < BCOL; ++u) {
          lo[u] = np;
          for (int r = 0; r < RB; ++r) acc[u][r] = (T)0;
        }
        col_dot_n<T, RB, BCOL>(pan + (int64_t)j0 * ld + a0, ld, ncol, a0, a0, lo, nf, xb, xld, lane, acc);
        for (int u = 0; u < ncol; ++u) {
          const int j = j0 + u;
          const T dj = pan[(int64_t)j * ld + j];
          for (int r = 0; r < nr; ++r) {
            const T t = warp_sum(acc[u][r]);
            if (lane == 0)
              TV[fv_off[tk.node] * nrhs + (int64_t)(r0 + r) * nf + j] =
                  X[P.vec_off * nrhs + (int64_t)(r0 + r) * P.n + N.p0 + j] / dj - t;
          }
        }
      }
      ex.sync();
    }
  }
};

// backward (2): x_p = L11^{-T} t for a task of pivot columns (warp per
// column, lanes along W-row vectors of the column below the diagonal)
template <class T, int RB>
struct KBwdPivots {
  BddcView V;
  const SolveTask* tasks;
  const T* F;
  const T* TV;
  const int64_t* fv_off;
  T* X;
  int nrhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    constexpr int W = VecW<T>::W;
    const SolveTask tk = tasks[blk];
    const NodeDev N = V.nodes[tk.node];
    const ProbDev P = V.probs[N.prob];
    const int np = N.np, nf = N.np + N.nb, ld = N.ld;
    const T* pan = F + N.panel_off;
    // rows tk.start..np-1 staged from the aligned row bs: ts[r*L + row - bs],
    // zero below tk.start and past np
    const int bs = (tk.start / W) * W;
    const int L = ((np - bs + W - 1) / W) * W;
    T* ts = reinterpret_cast<T*>(ex.smem);   // [RB][L]
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
      for (int q = ex.tid; q < RB * L; q += ex.nt) {
        const int r = q / L, row = bs + q % L;
        ts[q] = (r < nr && row >= tk.start && row < np)
                    ? TV[fv_off[tk.node] * nrhs + (int64_t)(r0 + r) * nf + row] : (T)0;
      }
      ex.sync();
      const int jend = tk.start + tk.count;
      for (int j0 = tk.start + BCOL * w; j0 < jend; j0 += BCOL * nw) {
        const int ncol = jend - j0 < BCOL ? jend - j0 : BCOL;
        const int b0 = ((j0 + 1) / W) * W;
        T acc[BCOL][RB];
        int lo[BCOL];
        for (int u = 0; u < BCOL; ++u) {
          lo[u] = j0 + u + 1;
          for (int r = 0; r < RB; ++r) acc[u][r] = (T)0;
        }
        col_dot_n<T, RB, BCOL>(pan + (int64_t)j0 * ld + b0, ld, ncol, b0, j0 + ncol, lo, np, ts + (b0 - bs), L,
                               lane, acc);
        for (int u = 0; u < ncol; ++u) {
          const int j = j0 + u;
          for (int r = 0; r < nr; ++r) {
            const T t = warp_sum(acc[u][r]);
            if (lane == 0)
              X[P.vec_off * nrhs + (int64_t)(r0 + r) * P.n + N.p0 + j] =
                  TV[fv_off[tk.node] * nrhs + (int64_t)(r0 + r) * nf + j] + t;
          }
        }
      }
      ex.sync();
    }
  }
};

// Residual of a local problem in FP64, R = B - K_q Z over the problem
// positions, in two deterministic steps.
//
// (1) KElemProduct: for each element of each problem of the batch, the
// element's share y_e = [A_e B_e^T; B_e 0] z_e of the product, with z_e
// gathered through the element's position map (entries outside the problem
// are zero).  One CTA per element: warps over the element's rows, lanes
// along the contiguous row of A_e (coalesced), RB right-hand sides per pass
// so every matrix entry read serves RB of them.  Output YE: per element
// (nK + np) rows for each right-hand side of the chunk.
//
// (2) KGatherResidual: per position, the sum of the element shares of its
// row in a fixed order (the subdomain's adjacency lists), the constraint
// terms of the constrained Neumann problem (multiplier columns and rows),
// and R = B - sum.
struct MatvecTask {
  int prob, start, count;
};
struct ElemTask {
  int prob, le;
};

// YE offset of element e's block for right-hand side r of a chunk of nr
VB_HD inline int64_t ye_off(const BddcView& V, int e, int nr, int r, int nKp) {
  return (V.offK[e] + (int64_t)V.np * e) * nr + (int64_t)r * nKp;
}

// x = hi + lo with hi = fl32(x), lo = fl32(x - hi): 48 significant bits
struct KSplitPairs {
  const double* x;
  float2* out;
  int64_t n;
  __device__ void operator()(const KExec& ex, int blk) const {
    const int64_t i = (int64_t)blk * ex.nt + ex.tid;
    if (i >= n) return;
    const double v = x[i];
    const float h = (float)v;
    out[i] = make_float2(h, (float)(v - (double)h));
  }
};

// double-float accumulation: (s, c) holds s + c with |c| << |s|;
// add a*b (a, b FP32) exactly up to the rounding of c (TwoProd with an FMA,
// TwoSum), plus the first-order low-part terms
// (the _rn intrinsics keep the compiler from contracting the error-free
// steps into FMAs)
__device__ inline void df_fma(float& s, float& c, float ah, float al, float zh, float zl) {
  const float p = __fmul_rn(ah, zh);
  const float e = fmaf(ah, zh, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c += err + e + fmaf(ah, zl, al * zh);
}
__device__ inline void df_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
  s = t;
  c += c2 + err;
}

// DF = true: the A_e part in double-float arithmetic on the FP32 units from
// the (high, low) copy V.A2 (FP64 units run at a small fraction of the FP32
// rate here); the B_e parts stay FP64
template <int RB, bool DF = false>
struct KElemProduct {
  BddcView V;
  const ElemTask* tasks;
  const double* Z;
  double* YE;
  int nrhs, r0, nr;   // chunk [r0, r0 + nr) of the nrhs right-hand sides
  __device__ void operator()(const KExec& ex, int blk) const {
    const ElemTask tk = tasks[blk];
    const ProbDev P = V.probs[tk.prob];
    const SubDev S = V.subs[P.sub];
    const int npk = V.np;
    const int e = V.sub_elems[S.elem_off + tk.le];
    const int nK = (int)(V.offK[e + 1] - V.offK[e]), nKp = nK + npk;
    const int* ep = V.elpos + P.elpos_off + V.elptr[P.elptr_off + tk.le];
    const double* Ae = V.A + V.offK2[e];
    const double* Be = V.B + (int64_t)npk * V.offK[e];
    double* zs = ex.smem;   // [RB][nKp]
    float* zf = reinterpret_cast<float*>(ex.smem + RB * nKp);   // DF: [RB][nKp] high, then low parts
    const int nw = ex.nt >> 5, w = ex.tid >> 5, lane = ex.tid & 31;
    for (int c0 = 0; c0 < nr; c0 += RB) {
      const int nc = nr - c0 < RB ? nr - c0 : RB;
      for (int q = ex.tid; q < RB * nKp; q += ex.nt) {
        const int r = q / nKp, b = q % nKp, x = ep[b];
        const double z = (r < nc && x >= 0) ? Z[P.vec_off * nrhs + (int64_t)(r0 + c0 + r) * P.n + x] : 0.0;
        zs[q] = z;
        if (DF) {
          const float h = (float)z;
          zf[q] = h;
          zf[RB * nKp + q] = (float)(z - (double)h);
        }
      }
      ex.sync();
      if (DF) {
        // velocity rows: one thread per row a, reading column a of the
        // symmetric A_e (consecutive threads, consecutive entries), eight
        // loads in flight per thread; no reductions
        for (int a = ex.tid; a < nK; a += ex.nt) {
          if (ep[a] < 0) continue;   // not a row of this problem
          float sh[RB], sl[RB];
          for (int r = 0; r < RB; ++r) sh[r] = sl[r] = 0.0f;
          const float2* col = V.A2 + V.offK2[e] + a;
          int b = 0;
          for (; b + 8 <= nK; b += 8) {
            float2 v[8];
            for (int u = 0; u < 8; ++u) v[u] = col[(int64_t)(b + u) * nK];
            for (int u = 0; u < 8; ++u)
              for (int r = 0; r < RB; ++r)
                df_fma(sh[r], sl[r], v[u].x, v[u].y, zf[r * nKp + b + u], zf[RB * nKp + r * nKp + b + u]);
          }
          for (; b < nK; ++b) {
            const float2 v = col[(int64_t)b * nK];
            for (int r = 0; r < RB; ++r)
              df_fma(sh[r], sl[r], v.x, v.y, zf[r * nKp + b], zf[RB * nKp + r * nKp + b]);
          }
          for (int r = 0; r < RB; ++r) {
            double acc = (double)sh[r] + (double)sl[r];
            for (int al = 0; al < npk; ++al) acc += Be[(int64_t)al * nK + a] * zs[r * nKp + nK + al];
            if (r < nc) YE[ye_off(V, e, nr, c0 + r, nKp) + a] = acc;
          }
        }
      }
      for (int a = DF ? nK + w : w; a < nKp; a += nw) {
        if (ep[a] < 0) continue;   // not a row of this problem
        double acc[RB];
        for (int r = 0; r < RB; ++r) acc[r] = 0.0;
        const double* row = a < nK ? Ae + (int64_t)a * nK : Be + (int64_t)(a - nK) * nK;
        if (DF && a < nK) {
          const float2* row2 = V.A2 + V.offK2[e] + (int64_t)a * nK;
          float sh[RB], sl[RB];
          for (int r = 0; r < RB; ++r) sh[r] = sl[r] = 0.0f;
          for (int b = lane; b < nK; b += 32) {
            const float2 v = row2[b];
            for (int r = 0; r < RB; ++r) df_fma(sh[r], sl[r], v.x, v.y, zf[r * nKp + b], zf[RB * nKp + r * nKp + b]);
          }
          for (int r = 0; r < RB; ++r) {
            for (int o = 16; o > 0; o >>= 1) {
              const float s2 = __shfl_xor_sync(0xffffffffu, sh[r], o), c2 = __shfl_xor_sync(0xffffffffu, sl[r], o);
              df_add(sh[r], sl[r], s2, c2);
            }
            // every lane holds the sum; lane 0 adds it once below
            if (lane == 0) acc[r] = (double)sh[r] + (double)sl[r];
          }
        } else {
          for (int b = lane; b < nK; b += 32) {
            const double v = row[b];
            for (int r = 0; r < RB; ++r) acc[r] += v * zs[r * nKp + b];
          }
        }
        if (a < nK)
          for (int al = lane; al < npk; al += 32) {
            const double v = Be[(int64_t)al * nK + a];
            for (int r = 0; r < RB; ++r) acc[r] += v * zs[r * nKp + nK + al];
          }
        for (int r = 0; r < RB; ++r) {
          const double t = warp_sum(acc[r]);
          if (lane == 0 && r < nc) YE[ye_off(V, e, nr, c0 + r, nKp) + a] = t;
        }
      }
      ex.sync();
    }
  }
};

struct KGatherResidual {
  BddcView V;
  const MatvecTask* tasks;
  const double* Bv;   // right-hand sides   [vec_off*nrhs + r*n + pos]
  const double* Z;    // current solutions
  const double* YE;   // element shares of the chunk
  double* R;
  const int* mcon_ptr;   // per subdomain: multiplier -> (local vdof, coef)
  const int* mcon_vdof;
  const double* mcon_coef;
  int nrhs, r0, nr;
  __device__ void operator()(const KExec& ex, int blk) const {
    const MatvecTask tk = tasks[blk];
    const ProbDev P = V.probs[tk.prob];
    const SubDev S = V.subs[P.sub];
    const int npk = V.np;
    const int* pv = V.pos_of_vdof + P.pv_off;
    for (int r = 0; r < nr; ++r) {
      const int64_t base = P.vec_off * nrhs + (int64_t)(r0 + r) * P.n;
      const double* z = Z + base;
      for (int pos = tk.start + ex.tid; pos < tk.start + tk.count; pos += ex.nt) {
        const int dt = V.dtype[P.pos_off + pos], src = V.dsrc[P.pos_off + pos];
        double acc = 0.0;
        if (dt == DT_VEL) {
          const int* vp = V.vadj_ptr + S.vadj_ptr_off;
          for (int q = vp[src]; q < vp[src + 1]; ++q) {
            const int le = V.vadj[S.vadj_off + 2 * q], a = V.vadj[S.vadj_off + 2 * q + 1];
            const int e = V.sub_elems[S.elem_off + le];
            const int nKp = (int)(V.offK[e + 1] - V.offK[e]) + npk;
            acc += YE[ye_off(V, e, nr, r, nKp) + a];
          }
          if (P.kind == PK_NEUMANN) {
            const int* cp = V.vcon_ptr + S.vcon_ptr_off;
            for (int q = cp[src]; q < cp[src + 1]; ++q)
              acc += V.vcon_coef[S.vcon_off + q] * z[P.mult0 + V.vcon_id[S.vcon_off + q]];
          }
        } else if (dt == DT_PRESS) {
          const int le = src / npk, a = src % npk;
          const int e = V.sub_elems[S.elem_off + le];
          const int nK = (int)(V.offK[e + 1] - V.offK[e]);
          acc = YE[ye_off(V, e, nr, r, nK + npk) + nK + a];
        } else if (dt == DT_MULT) {
          const int* mp = mcon_ptr + S.mcon_ptr_off;
          for (int q = mp[src]; q < mp[src + 1]; ++q)
            acc += mcon_coef[S.mcon_off + q] * z[pv[mcon_vdof[S.mcon_off + q]]];
        }
        R[base + pos] = Bv[base + pos] - acc;
      }
    }
  }
};

}  // namespace vb

// BDDC preconditioner (Eq. BDDCprec) and PCG on the GPU: setup (local
// factorizations, deluxe face blocks, coarse basis and coarse matrix) and the
// per-iteration apply: restriction with the change of basis and scaling,
// coarse solve, constrained Neumann solves, averaging, Dirichlet harmonic
// extension.
#include "system.h"
#include "bddc_setup.h"
#include "bddc_dev.h"
#include "mf.cuh"
#include "dense.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <cstdio>
#include <numeric>
#include <chrono>
#include <map>
#include <tuple>
#include <utility>
#include <string>
#include <type_traits>

namespace vb {
void spmv(vem_system* s, const double* x, double* y, cudaStream_t st);
struct DelTask {
  int macro, k0;
};
struct IfTask {
  int sub, l0;
};

// one batch of problems (all Dirichlet, all Neumann or all deluxe ones)
struct Batch {
  std::vector<int> probs;                 // global problem ids
  int64_t vec_n = 0;                      // sum of problem sizes
  int64_t uvec_n = 0;                     // sum of border sizes
  int maxh = 0, maxnf = 0;
  std::vector<int> level_ptr;             // nodes grouped by height
  DBuf<int> d_levels;
  std::vector<int> h_levels;
  DBuf<double> F;                         // panels (FP64 local factors)
  DBuf<double> U;                         // update matrices
  DBuf<float> F32, U32;                   // the same in FP32 (FP32-local factors)
  DBuf<double> XB, XR;                    // refinement: right-hand sides, residuals
  std::vector<MatvecTask> h_mtask;
  DBuf<MatvecTask> d_mtask;
  std::vector<ElemTask> h_etask;          // (problem, local element) of every problem
  DBuf<ElemTask> d_etask;
  DBuf<double> YE;                        // element shares of the residual
  int64_t ye_n = 0;                       // per right-hand side
  int64_t nF = 0, nU = 0;
  int64_t nfv = 0;                        // sum of front sizes (front-vector store per rhs)
  std::vector<int> ptask_ptr, btask_ptr, fptask_ptr;   // per level: task ranges
  std::vector<SolveTask> h_ptask, h_btask, h_fptask;  // pivot columns, border vectors, pivot-row vectors
  DBuf<SolveTask> d_ptask, d_btask, d_fptask;
  DBuf<double> FV;
  int fv_nrhs = 0;
  DBuf<float> XF;                         // FP32 sweeps: right-hand sides and solutions in FP32
};

}  // namespace vb

struct bddc {
  vem_system* sys = nullptr;
  vb::BddcHost H;
  cudaStream_t stream = 0;
  vb::SetupOptions opt;
  int prec = 0;                  // 0 FP64 local factors; 1 FP32 + refinement; 2 FP32 plain
  int refine = 1;                // refinement steps of the FP32-local solves
  // device copies of the structure
  vb::DBuf<vb::NodeDev> d_nodes;
  vb::DBuf<int> d_mcon_ptr, d_mcon_vdof;
  vb::DBuf<double> d_mcon_coef;
  vb::DBuf<vb::ProbDev> d_probs;
  vb::DBuf<vb::SubDev> d_subs;
  vb::DBuf<vb::MacroDev> d_macros;
  vb::DBuf<int> d_border, d_children, d_rel, d_dtype, d_dsrc, d_bgrp, d_elpos, d_elptr, d_pv, d_sub_elems, d_vadj_ptr,
      d_vadj, d_vcon_ptr, d_vcon_id, d_iface, d_elloc, d_elloc_ptr, d_share, d_gpos, d_gif;
  vb::DBuf<int64_t> d_vdof, d_press, d_coarse, d_mdofs, d_fvoff;
  std::vector<int64_t> h_fvoff;
  vb::DBuf<double> d_vcon_coef, d_wmean, d_hv, d_tau, d_deluxe, d_deluxe_e;
  std::vector<vb::NodeDev> h_nodes;
  std::vector<vb::ProbDev> h_probs;
  std::vector<vb::SubDev> h_subs;
  std::vector<vb::MacroDev> h_macros;
  vb::Batch bd, bn, bx;          // Dirichlet, Neumann, deluxe batches
  // coarse
  int64_t nc = 0, ncv = 0;
  vb::DBuf<double> d_Kinv;       // inverse of the bordered coarse matrix, (nc+1)^2
  vb::DBuf<double> d_phi;        // Phi_Gamma per subdomain
  int64_t nphi = 0;
  vb::DBuf<int> d_cg_ptr, d_cg_sub, d_cg_loc;   // coarse row -> (subdomain, local coordinate)
  // apply workspaces
  vb::DBuf<double> XD, XN, UVD, UVN, rC, uC, cloc, wloc, dwork, y, part, dtw, wd1, avgd;
  std::vector<vb::DelTask> h_dtT, h_dtN;
  std::vector<vb::IfTask> h_ift;
  vb::DBuf<vb::DelTask> d_dtT, d_dtN;
  vb::DBuf<vb::IfTask> d_ift;
  int NC = 1;
  int max_nd = 1;
  int64_t ndual = 0, niface_tot = 0;
  // PCG vectors
  vb::DBuf<double> r, z, p, Ap, scal;
  std::vector<std::pair<std::string, double>> times;   // setup phase wall times (ms)
  // CUDA graphs: the PCG loop (one conditional while node whose body is one
  // iteration) and bddc_apply; captured on a private stream, replayed on
  // `stream`
  bool use_graph = true;
  vb::DBuf<float2> d_A2;         // element matrices as FP32 pairs (FP32-local refinement residual)
  bool use_tc = false;           // FP32 front updates on the tensor cores (tcgen05, split TF32)
  // adaptive coarse space (Sec. 6): threshold, rows added, and the face
  // Schur complements S_F kept from the first setup
  double adapt_theta = 0.0;
  int n_adaptive = 0;
  bool keep_sf = false;
  vb::DBuf<double> d_sf;
  std::vector<int> sf_faces;
  std::vector<int64_t> sf_i, sf_j;
  cudaStream_t cap_stream = nullptr;
  vb::DBuf<double> xg, pcg_s, pcg_al, pcg_be;   // iterate, scalars, Lanczos records
  int pcg_cap = 0;                              // records allocated (>= maxit)
  cudaGraphExec_t pcg_exec = nullptr;
  int64_t pcg_body_launches = 0;
  cudaGraphExec_t app_exec = nullptr;
  const double* app_r = nullptr;
  double* app_z = nullptr;
  int64_t app_launches = 0;
  ~bddc() {
    if (pcg_exec) cudaGraphExecDestroy(pcg_exec);
    if (app_exec) cudaGraphExecDestroy(app_exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace vb {

static BddcView make_view(bddc* b) {
  vem_system* s = b->sys;
  BddcView V{};
  V.np = s->dof.np;
  V.k = s->dof.k;
  V.nvf = s->dof.nvf;
  V.n = s->n;
  V.offK = s->d_eoff.p;
  V.offK2 = s->d_eoffK2.p;
  V.A = s->d_A.p;
  V.A2 = b->d_A2.p;
  V.B = s->d_B.p;
  V.nodes = b->d_nodes.p;
  V.probs = b->d_probs.p;
  V.subs = b->d_subs.p;
  V.macros = b->d_macros.p;
  V.border = b->d_border.p;
  V.children = b->d_children.p;
  V.rel = b->d_rel.p;
  V.dtype = b->d_dtype.p;
  V.dsrc = b->d_dsrc.p;
  V.bgrp = b->d_bgrp.p;
  V.elpos = b->d_elpos.p;
  V.elptr = b->d_elptr.p;
  V.pos_of_vdof = b->d_pv.p;
  V.sub_elems = b->d_sub_elems.p;
  V.vdof = b->d_vdof.p;
  V.vadj_ptr = b->d_vadj_ptr.p;
  V.vadj = b->d_vadj.p;
  V.vcon_ptr = b->d_vcon_ptr.p;
  V.vcon_id = b->d_vcon_id.p;
  V.vcon_coef = b->d_vcon_coef.p;
  V.press = b->d_press.p;
  V.wmean = b->d_wmean.p;
  V.iface = b->d_iface.p;
  V.coarse = b->d_coarse.p;
  V.elloc = b->d_elloc.p;
  V.elloc_ptr = b->d_elloc_ptr.p;
  V.mdofs = b->d_mdofs.p;
  V.hv = b->d_hv.p;
  V.tau = b->d_tau.p;
  V.share = b->d_share.p;
  V.gpos = b->d_gpos.p;
  V.gif = b->d_gif.p;
  V.deluxe = b->d_deluxe.p;
  V.deluxe_e = b->d_deluxe_e.p;
  V.ncv = b->ncv;
  V.nc = b->nc;
  return V;
}

// ----------------------------------------------------------------- helpers

// c = H^T v (in place) with the r reflectors of entity G (n values)
VB_HD inline void hh_T_inplace(const BddcView& V, const MacroDev& G, double* c) {
  for (int q = 0; q < G.r; ++q) {
    if (G.hv_off < 0) break;
    const double* h = V.hv + G.hv_off + (int64_t)q * G.n;
    double dot = 0.0;
    for (int i = 0; i < G.n; ++i) dot += h[i] * c[i];
    dot *= V.tau[G.tau_off + q];
    for (int i = 0; i < G.n; ++i) c[i] -= dot * h[i];
  }
}
VB_HD inline void hh_inplace(const BddcView& V, const MacroDev& G, double* c) {
  for (int q = G.r - 1; q >= 0; --q) {
    if (G.hv_off < 0) break;
    const double* h = V.hv + G.hv_off + (int64_t)q * G.n;
    double dot = 0.0;
    for (int i = 0; i < G.n; ++i) dot += h[i] * c[i];
    dot *= V.tau[G.tau_off + q];
    for (int i = 0; i < G.n; ++i) c[i] -= dot * h[i];
  }
}

// Column-major subdomain blocks (entry (row, c) of subdomain i at
// loc_off*NC + c*nloc + row) to one row-major array over all local rows
// (global local row g = loc_off + row at g*NC + c); DF: as FP32 (high, low)
// pairs.  One CTA per 32 consecutive local rows, NC in tiles of 32.
template <bool DF>
struct KToRowMajor {
  const int64_t* row_ptr;   // prefix of nloc over subdomains
  int nsub;
  int64_t loc;
  const double* X;
  void* Y;
  int NC;
  __device__ void operator()(const KExec& ex, int blk) const {
    double* tile = ex.smem;   // [32][33]
    const int tr = ex.tid & 31, tc = ex.tid >> 5, ntc = ex.nt >> 5;
    const int64_t g = (int64_t)blk * 32 + tr;
    int lo = 0, hi = nsub - 1;
    if (g < loc)
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (row_ptr[mid] <= g) lo = mid; else hi = mid - 1;
      }
    const int64_t off = row_ptr[lo], nloc = row_ptr[lo + 1] - off;
    for (int c0 = 0; c0 < NC; c0 += 32) {
      for (int c = tc; c < 32; c += ntc)
        tile[tr * 33 + c] = (g < loc && c0 + c < NC) ? X[off * NC + (int64_t)(c0 + c) * nloc + (g - off)] : 0.0;
      ex.sync();
      for (int r = tc; r < 32; r += ntc) {
        const int64_t gr = (int64_t)blk * 32 + r;
        if (gr >= loc || c0 + tr >= NC) continue;
        const double v = tile[r * 33 + tr];
        if (DF) {
          const float h = (float)v;
          reinterpret_cast<float2*>(Y)[gr * NC + c0 + tr] = make_float2(h, (float)(v - (double)h));
        } else {
          reinterpret_cast<double*>(Y)[gr * NC + c0 + tr] = v;
        }
      }
      ex.sync();
    }
  }
};

// Y = K_i X on the subdomain-local dense blocks, X and Y row-major over all
// local rows (row g at g*NC; local velocity DOFs, then local pressures).
// One warp per row, each lane 4 columns of a 128-column block, so that every
// load of X serves the 32 lanes from consecutive addresses.  DF: X given as
// FP32 (high, low) pairs and the A_e terms in double-float arithmetic on the
// FP32 units from V.A2; the B_e terms stay FP64.
template <bool DF>
struct KElemMatvecRM {
  BddcView V;
  const int64_t* row_ptr;
  int nsub;
  const void* X;
  double* Y;
  int NC;
  __device__ double xval(int64_t i) const {
    if (DF) {
      const float2 x = reinterpret_cast<const float2*>(X)[i];
      return (double)x.x + (double)x.y;
    }
    return reinterpret_cast<const double*>(X)[i];
  }
  __device__ void operator()(const KExec& ex, int blk) const {
    int lo = 0, hi = nsub - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (row_ptr[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    const SubDev S = V.subs[lo];
    const int row = (int)(blk - row_ptr[lo]);
    const int64_t xb = S.loc_off * NC;   // row l of the subdomain at xb + l*NC
    const int npk = V.np;
    const int* ellp = V.elloc_ptr + S.ellocptr_off;
    const int lane = ex.tid;
    for (int cb = 0; cb < NC; cb += 128) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
      bool ok[4];
      for (int j = 0; j < 4; ++j) ok[j] = cb + lane + 32 * j < NC;
      if (row < S.nv) {
        const int* vp = V.vadj_ptr + S.vadj_ptr_off;
        for (int q = vp[row]; q < vp[row + 1]; ++q) {
          const int le = V.vadj[S.vadj_off + 2 * q], a = V.vadj[S.vadj_off + 2 * q + 1];
          const int e = V.sub_elems[S.elem_off + le];
          const int nK = (int)(V.offK[e + 1] - V.offK[e]);
          const double* Be = V.B + (int64_t)npk * V.offK[e];
          const int* el = V.elloc + S.elloc_off + ellp[le];
          if (DF) {
            const float2* Ae2 = V.A2 + V.offK2[e] + (int64_t)a * nK;
            for (int b = 0; b < nK; ++b) {
              const int l = el[b];
              if (l < 0) continue;
              const float2 v = Ae2[b];
              const float2* xr = reinterpret_cast<const float2*>(X) + xb + (int64_t)l * NC + cb + lane;
              for (int j = 0; j < 4; ++j)
                if (ok[j]) {
                  const float2 x = xr[32 * j];
                  df_fma(sh[j], sl[j], v.x, v.y, x.x, x.y);
                }
            }
          } else {
            const double* Ae = V.A + V.offK2[e] + (int64_t)a * nK;
            for (int b = 0; b < nK; ++b) {
              const int l = el[b];
              if (l < 0) continue;
              const double v = Ae[b];
              const double* xr = reinterpret_cast<const double*>(X) + xb + (int64_t)l * NC + cb + lane;
              for (int j = 0; j < 4; ++j)
                if (ok[j]) acc[j] += v * xr[32 * j];
            }
          }
          for (int b = nK; b < nK + npk; ++b) {
            const int l = el[b];
            if (l < 0) continue;
            const double v = Be[(int64_t)(b - nK) * nK + a];
            for (int j = 0; j < 4; ++j)
              if (ok[j]) acc[j] += v * xval(xb + (int64_t)l * NC + cb + lane + 32 * j);
          }
        }
      } else {
        const int q = row - S.nv;
        const int le = q / npk, a = q % npk;
        const int e = V.sub_elems[S.elem_off + le];
        const int nK = (int)(V.offK[e + 1] - V.offK[e]);
        const double* Be = V.B + (int64_t)npk * V.offK[e];
        const int* el = V.elloc + S.elloc_off + ellp[le];
        for (int b = 0; b < nK; ++b) {
          const int l = el[b];
          if (l < 0) continue;
          const double v = Be[(int64_t)a * nK + b];
          for (int j = 0; j < 4; ++j)
            if (ok[j]) acc[j] += v * xval(xb + (int64_t)l * NC + cb + lane + 32 * j);
        }
      }
      for (int j = 0; j < 4; ++j)
        if (ok[j]) Y[xb + (int64_t)row * NC + cb + lane + 32 * j] = acc[j] + (DF ? (double)sh[j] + (double)sl[j] : 0.0);
    }
  }
};

// Y = K_i W for the coarse basis before its Neumann correction.  Row l of W
// is nonzero only in the columns [wcols[l].x, wcols[l].x + wcols[l].y): the
// primal coordinates of the entity holding interface DOF l, or the p_0
// column at a constant pressure coefficient.  One warp per row walks the
// row's element entries in the order of the dense product (element, then
// column) and adds only the terms whose W row is nonzero, so every column
// sums the same nonzero terms in the same order as K_i W formed densely.
// Y must be cleared beforehand: rows without such terms are not written.
struct KElemMatvecW {
  BddcView V;
  const int64_t* row_ptr;   // prefix of nloc over subdomains
  int nsub;
  const double* X;
  const int2* wcols;        // per local row at loc_off: first column, count
  double* Y;
  int NC;
  __device__ void operator()(const KExec& ex, int blk) const {
    int lo = 0, hi = nsub - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (row_ptr[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    const SubDev S = V.subs[lo];
    const int nloc = S.nv + S.npress;
    const int row = (int)(blk - row_ptr[lo]);
    const double* Xs = X + S.loc_off * NC;
    const int2* wc = wcols + S.loc_off;
    const int npk = V.np;
    const int* ellp = V.elloc_ptr + S.ellocptr_off;
    const int lane = ex.tid;
    double* acc = ex.smem;   // [NC]
    for (int c = lane; c < NC; c += 32) acc[c] = 0.0;
    bool any = false;
    // the entries [0, nb) of one element row: coefficient coef(b), local index el[b]
    auto walk = [&](const int* el, int nb, auto coef) {
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        const int l = b < nb ? el[b] : -1;
        const int2 w = l >= 0 ? wc[l] : make_int2(0, 0);
        const double v = w.y > 0 ? coef(b) : 0.0;
        unsigned m = __ballot_sync(0xffffffffu, w.y > 0);
        any |= m != 0;
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int ls = __shfl_sync(0xffffffffu, l, src);
          const int c0 = __shfl_sync(0xffffffffu, w.x, src), cn = __shfl_sync(0xffffffffu, w.y, src);
          const double vs = __shfl_sync(0xffffffffu, v, src);
          __syncwarp();
          for (int t = lane; t < cn; t += 32) acc[c0 + t] += vs * Xs[(int64_t)(c0 + t) * nloc + ls];
        }
      }
    };
    if (row < S.nv) {
      const int* vp = V.vadj_ptr + S.vadj_ptr_off;
      for (int q = vp[row]; q < vp[row + 1]; ++q) {
        const int le = V.vadj[S.vadj_off + 2 * q], a = V.vadj[S.vadj_off + 2 * q + 1];
        const int e = V.sub_elems[S.elem_off + le];
        const int nK = (int)(V.offK[e + 1] - V.offK[e]);
        const double* Ae = V.A + V.offK2[e];
        const double* Be = V.B + (int64_t)npk * V.offK[e];
        walk(V.elloc + S.elloc_off + ellp[le], nK + npk, [&](int b) {
          return b < nK ? Ae[(int64_t)a * nK + b] : Be[(int64_t)(b - nK) * nK + a];
        });
      }
    } else {
      const int q = row - S.nv;
      const int le = q / npk, a = q % npk;
      const int e = V.sub_elems[S.elem_off + le];
      const int nK = (int)(V.offK[e + 1] - V.offK[e]);
      const double* Be = V.B + (int64_t)npk * V.offK[e];
      walk(V.elloc + S.elloc_off + ellp[le], nK, [&](int b) { return Be[(int64_t)a * nK + b]; });
    }
    __syncwarp();
    if (!any) return;
    double* Ys = Y + S.loc_off * NC;
    for (int c = lane; c < NC; c += 32) Ys[(int64_t)c * nloc + row] = acc[c];
  }
};

// Neumann right-hand sides of the coarse basis: -K W at the problem
// positions, pressure part projected onto sum-zero data (zero-mean Q_I)
// (columns c0 .. c0+ch-1 of the NC coarse columns; XN holds ch columns)
struct KNeuRhsPhi {
  BddcView V;
  const double* KW;
  double* XN;
  int NC, c0, ch;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int i = blk / ch, c = blk % ch;
    const SubDev S = V.subs[i];
    const ProbDev P = V.probs[S.neu];
    const int nloc = S.nv + S.npress;
    const double* kw = KW + S.loc_off * NC + (int64_t)(c0 + c) * nloc;
    double* x = XN + P.vec_off * ch + (int64_t)c * P.n;
    // compatibility with the subdomain-constant pressure: shift the pressure
    // data by (sum of its constant-coefficient entries)/|Omega_i| times w
    double sg = 0.0;
    for (int le = ex.tid; le < S.ne; le += ex.nt) sg -= kw[S.nv + le * V.np];
    sg = block_sum(ex, sg, ex.smem);
    const double shift = sg / S.wsum;
    for (int pos = ex.tid; pos < P.n; pos += ex.nt) {
      const int dt = V.dtype[P.pos_off + pos], src = V.dsrc[P.pos_off + pos];
      double v = 0.0;
      if (dt == DT_VEL) v = -kw[src];
      else if (dt == DT_PRESS) v = -kw[S.nv + src] - shift * V.wmean[S.press_off + src];
      x[pos] = v;
    }
  }
};

// Phi = W + Z (local layout); Z read from the Neumann solution, its
// pressure made zero-mean
struct KPhiAssemble {
  BddcView V;
  const double* W;
  const double* XN;
  double* PHI;
  int NC, c0, ch;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int i = blk / ch, c = blk % ch;
    const SubDev S = V.subs[i];
    const ProbDev P = V.probs[S.neu];
    const int nloc = S.nv + S.npress;
    const double* w = W + S.loc_off * NC + (int64_t)(c0 + c) * nloc;
    double* phi = PHI + S.loc_off * NC + (int64_t)(c0 + c) * nloc;
    const double* x = XN + P.vec_off * ch + (int64_t)c * P.n;
    const int* pv = V.pos_of_vdof + P.pv_off;
    for (int v = ex.tid; v < S.nv; v += ex.nt) {
      const int pos = pv[v];
      phi[v] = w[v] + (pos >= 0 ? x[pos] : 0.0);
    }
    // pressures: position via the element table of the problem
    double wp = 0.0;
    const int npk = V.np;
    for (int q = ex.tid; q < S.npress; q += ex.nt) {
      const int le = q / npk, a = q % npk;
      const int e = V.sub_elems[S.elem_off + le];
      const int nK = (int)(V.offK[e + 1] - V.offK[e]);
      const int pos = V.elpos[P.elpos_off + V.elptr[P.elptr_off + le] + nK + a];
      const double pz = pos >= 0 ? x[pos] : 0.0;
      phi[S.nv + q] = pz;
      wp += V.wmean[S.press_off + q] * pz;
    }
    wp = block_sum(ex, wp, ex.smem);
    const double m = wp / S.wsum;   // remove m * 1_{Omega_i}: constant coefficients only
    for (int q = ex.tid; q < S.npress; q += ex.nt) phi[S.nv + q] += w[S.nv + q] - (q % npk == 0 ? m : 0.0);
  }
};

// S_Pi = Phi^T (K Phi) per subdomain by 32 x 32 output tiles: one CTA per
// (subdomain, tile), 256 threads with 4 outputs each, the rows streamed in
// chunks of 64 through shared memory; every entry sums the rows in order.
struct GramTile {
  int sub, a0, b0;
};
struct KGramTiled {
  BddcView V;
  const GramTile* tiles;
  const double* PHI;    // column-major subdomain blocks
  const double* KPHI;   // row-major over all local rows (row g at g*NC)
  double* SG;
  int NC;
  static constexpr int TR = 64, TP = 33;   // rows per chunk, padded tile width
  VB_HD void operator()(const KExec& ex, int blk) const {
    const GramTile tl = tiles[blk];
    const SubDev S = V.subs[tl.sub];
    const int nloc = S.nv + S.npress, ncl = S.ncl;
    const double* ph = PHI + S.loc_off * NC;
    const double* kp = KPHI + S.loc_off * NC;   // row l at l*NC
    double* sA = ex.smem;            // [TR][TP]: Phi rows, columns a0 ..
    double* sB = sA + TR * TP;       // [TR][TP]: K Phi rows, columns b0 ..
    const int a = ex.tid / 8, bq = (ex.tid % 8) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = 0; r0 < nloc; r0 += TR) {
      const int nr = nloc - r0 < TR ? nloc - r0 : TR;
      for (int q = ex.tid; q < TR * 32; q += ex.nt) {
        const int c = q / TR, r = q % TR;
        sA[r * TP + c] = (r < nr && tl.a0 + c < ncl) ? ph[(int64_t)(tl.a0 + c) * nloc + r0 + r] : 0.0;
        const int c2 = q % 32, r2 = q / 32;
        sB[r2 * TP + c2] = (r2 < nr && tl.b0 + c2 < ncl) ? kp[(int64_t)(r0 + r2) * NC + tl.b0 + c2] : 0.0;
      }
      ex.sync();
      for (int r = 0; r < nr; ++r) {
        const double x = sA[r * TP + a];
        for (int j = 0; j < 4; ++j) acc[j] += x * sB[r * TP + bq + j];
      }
      ex.sync();
    }
    if (tl.a0 + a < ncl)
      for (int j = 0; j < 4; ++j)
        if (tl.b0 + bq + j < ncl) SG[(int64_t)tl.sub * NC * NC + (tl.a0 + a) * NC + tl.b0 + bq + j] = acc[j];
  }
};

// interface rows of Phi (velocity part), column-major niface x ncl
struct KPhiGamma {
  BddcView V;
  const double* PHI;
  double* PG;
  int NC;
  VB_HD void operator()(const KExec& ex, int i) const {
    const SubDev S = V.subs[i];
    const int nloc = S.nv + S.npress;
    const double* ph = PHI + S.loc_off * NC;
    for (int idx = ex.tid; idx < S.niface * S.ncl; idx += ex.nt) {
      const int c = idx / S.niface, l = idx % S.niface;
      PG[S.phi_off + idx] = ph[(int64_t)c * nloc + V.iface[S.iface_off + l]];
    }
  }
};

// bordered coarse matrix (one CTA, subdomains in order: deterministic sums)
struct KCoarseAssemble {
  BddcView V;
  const double* SG;
  double* KB;
  int N, NC;
  VB_HD void operator()(const KExec& ex, int) const {
    const int64_t nb = V.nc + 1;
    for (int64_t q = ex.tid; q < nb * nb; q += ex.nt) KB[q] = 0.0;
    ex.sync();
    for (int i = 0; i < N; ++i) {
      const SubDev S = V.subs[i];
      const int64_t* g = V.coarse + S.coarse_off;
      for (int idx = ex.tid; idx < S.ncl * S.ncl; idx += ex.nt) {
        const int a = idx / S.ncl, b = idx % S.ncl;
        KB[g[a] * nb + g[b]] += SG[(int64_t)i * NC * NC + a * NC + b];
      }
      ex.sync();
      if (ex.tid == 0) {
        KB[(V.ncv + i) * nb + V.nc] = S.volume;
        KB[V.nc * nb + V.ncv + i] = S.volume;
      }
      ex.sync();
    }
  }
};

// Dirichlet factors from the deluxe factorization: the deluxe problem of a
// subdomain has the Dirichlet problem's pivots, in the same order and tree,
// and every front's border is the Dirichlet border followed by entity DOFs
// (positions beyond all pivots).  Its panels therefore hold the Dirichlet
// panels as their first np + nb_D rows (L11^{-1} in place, D, L21): copied,
// one CTA per (node pair, 32 columns), the padding rows up to the leading
// dimension zero as after a factorization.
struct PanelCopyTask {
  int dst, src, c0;   // Dirichlet node, deluxe node, first column
};
template <class T>
struct KPanelCopy {
  BddcView V;
  const PanelCopyTask* tasks;
  const T* FX;   // deluxe factor store
  T* FD;         // Dirichlet factor store
  VB_HD void operator()(const KExec& ex, int blk) const {
    const PanelCopyTask tk = tasks[blk];
    const NodeDev D = V.nodes[tk.dst], X = V.nodes[tk.src];
    const int rows = D.np + D.nb;
    const int c1 = tk.c0 + 32 < D.np ? tk.c0 + 32 : D.np;
    for (int c = tk.c0; c < c1; ++c) {
      const T* src = FX + X.panel_off + (int64_t)c * X.ld;
      T* dst = FD + D.panel_off + (int64_t)c * D.ld;
      for (int r = ex.tid; r < D.ld; r += ex.nt) dst[r] = r < rows ? src[r] : (T)0;   // padding rows zero
    }
  }
};

// deluxe: S_FF of one side from the root update matrix of its subdomain's
// deluxe problem (the entity's DOFs are the contiguous root-border block
// b0 .. b0 + n), rotated to the dual coordinates: Sd = (H^T S H)[r:, r:]
struct DeluxeTask {
  int prob, root, macro, b0;
  int64_t work_off, sd_off;
};

template <class T>
struct KDeluxeExtract {
  BddcView V;
  const DeluxeTask* tasks;
  const T* U;             // deluxe batch update store
  double* work;           // n x n per task
  double* SD;             // dual blocks
  VB_HD void operator()(const KExec& ex, int blk) const {
    const DeluxeTask tk = tasks[blk];
    const NodeDev R = V.nodes[tk.root];
    const MacroDev F = V.macros[tk.macro];
    const int n = F.n, r = F.r, nd = n - r, nbU = R.nb, b0 = tk.b0;
    const T* Ur = U + R.upd_off;
    double* S = work + tk.work_off;
    for (int64_t idx = ex.tid; idx < (int64_t)n * n; idx += ex.nt) {
      const int k = (int)(idx / n), i = (int)(idx % n);
      S[idx] = (double)(i >= k ? Ur[(int64_t)(b0 + k) * nbU + b0 + i] : Ur[(int64_t)(b0 + i) * nbU + b0 + k]);
    }
    ex.sync();
    // S <- H^T S (columns), then S <- (H^T S^T)^T = H^T S H using symmetry of S
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < r; ++q) {
        const double* h = V.hv + F.hv_off + (int64_t)q * n;
        const double tau = V.tau[F.tau_off + q];
        for (int j = ex.tid; j < n; j += ex.nt) {
          double* col = S + (int64_t)j * n;
          double dot = 0.0;
          for (int i = 0; i < n; ++i) dot += h[i] * col[i];
          dot *= tau;
          for (int i = 0; i < n; ++i) col[i] -= dot * h[i];
        }
        ex.sync();
      }
      // transpose in place
      for (int64_t idx = ex.tid; idx < (int64_t)n * n; idx += ex.nt) {
        const int k = (int)(idx / n), i = (int)(idx % n);
        if (i > k) { double t = S[(int64_t)k * n + i]; S[(int64_t)k * n + i] = S[(int64_t)i * n + k]; S[(int64_t)i * n + k] = t; }
      }
      ex.sync();
    }
    double* sd = SD + tk.sd_off;
    for (int64_t idx = ex.tid; idx < (int64_t)nd * nd; idx += ex.nt) {
      const int k = (int)(idx / nd), i = (int)(idx % nd);
      sd[idx] = 0.5 * (S[(int64_t)(r + k) * n + r + i] + S[(int64_t)(r + i) * n + r + k]);
    }
  }
};

// deluxe via a dense front: partial LDL^T of [[S_i + S_j, .], [S_i, .]]
// gives L21 = S_i L11^{-T} Dg^{-1}, hence D^T = S_i (S_i+S_j)^{-1} = L21 L11^{-1}
struct KDeluxeFront {
  BddcView V;
  const int* faces;
  const int64_t* sd_i;
  const int64_t* sd_j;
  const double* SD;
  double* PAN;
  double* UPD;
  const int64_t* pan_off;
  const int64_t* upd_off;
  int* status;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const MacroDev F = V.macros[faces[blk]];
    const int nd = F.ndual, nf = 2 * nd;
    const double* Si = SD + sd_i[blk];
    const double* Sj = SD + sd_j[blk];
    double* pan = PAN + pan_off[blk];
    double* upd = UPD + upd_off[blk];
    for (int64_t idx = ex.tid; idx < (int64_t)nd * nf; idx += ex.nt) {
      const int j = (int)(idx / nf), i = (int)(idx % nf);
      pan[idx] = i < nd ? Si[(int64_t)j * nd + i] + Sj[(int64_t)j * nd + i] : Si[(int64_t)j * nd + (i - nd)];
    }
    for (int64_t idx = ex.tid; idx < (int64_t)nd * nd; idx += ex.nt) upd[idx] = 0.0;
    ex.sync();
    // only L21 = S_i L11^{-T} Dg^{-1} is used: the border block is not formed
    front_ldlt<double>(ex, pan, upd, nd, nd, nf, nullptr, status, nullptr, FrontGroups{nullptr, nullptr, 0}, false);
  }
};

// deluxe on macro edges (scaling 2): W = sum of the dual blocks S_s of the
// subdomains sharing the edge, one CTA per edge
struct KDeluxeEdgeSum {
  BddcView V;
  const int* edges;
  const int64_t* sd_ptr;   // per edge: first of its blocks in sd_off
  const int64_t* sd_off;   // offsets of the blocks S_s in SD, sharing-list order
  const double* SD;
  double* W;
  const int64_t* w_off;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const MacroDev G = V.macros[edges[blk]];
    const int64_t nn = (int64_t)G.ndual * G.ndual;
    const int64_t* so = sd_off + sd_ptr[blk];
    double* w = W + w_off[blk];
    for (int64_t idx = ex.tid; idx < nn; idx += ex.nt) {
      double acc = 0.0;
      for (int s = 0; s < G.nshare; ++s) acc += SD[so[s] + idx];
      w[idx] = acc;
    }
  }
};

// D_s = W^{-1} S_s with the Cholesky factor W = G G^T (lower, column-major):
// one CTA per (edge, sharing subdomain), one column of S_s per thread
// (forward then backward substitution in place in the output column)
struct KDeluxeEdgeSolve {
  BddcView V;
  const int* edges;
  const int* task_edge;
  const int* task_share;
  const int64_t* sd_ptr;
  const int64_t* sd_off;
  const double* SD;
  const double* W;
  const int64_t* w_off;
  double* DE;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int t = task_edge[blk], q = task_share[blk];
    const MacroDev G = V.macros[edges[t]];
    const int nd = G.ndual;
    const double* L = W + w_off[t];
    const double* S = SD + sd_off[sd_ptr[t] + q];
    double* D = DE + G.deluxe_e_off + (int64_t)q * nd * nd;
    for (int c = ex.tid; c < nd; c += ex.nt) {
      double* x = D + (int64_t)c * nd;
      for (int i = 0; i < nd; ++i) x[i] = S[(int64_t)c * nd + i];
      for (int j = 0; j < nd; ++j) {
        const double xj = x[j] / L[(int64_t)j * nd + j];
        x[j] = xj;
        for (int i = j + 1; i < nd; ++i) x[i] -= L[(int64_t)j * nd + i] * xj;
      }
      for (int j = nd - 1; j >= 0; --j) {
        double acc = x[j];
        for (int i = j + 1; i < nd; ++i) acc -= L[(int64_t)j * nd + i] * x[i];
        x[j] = acc / L[(int64_t)j * nd + j];
      }
    }
  }
};

struct GemmTile {
  int face, ti, tj;
};

// D (column-major) = (L21 L11^{-1})^T, 64 x 64 output tiles, k staged by 32
struct KDeluxeGemm {
  BddcView V;
  const GemmTile* tiles;
  const int* faces;
  const double* PAN;
  const int64_t* pan_off;
  double* DEL;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const GemmTile gt = tiles[blk];
    const MacroDev F = V.macros[faces[gt.face]];
    const int nd = F.ndual, nf = 2 * nd;
    const double* pan = PAN + pan_off[gt.face];
    double* D = DEL + F.deluxe_off;
    const int i0 = gt.ti * 64, j0 = gt.tj * 64;
    double* sA = ex.smem;            // [32][64]  L21 rows i0.., columns k
    double* sB = ex.smem + 32 * 64;  // [32][64]  Linv rows k, columns j0..
    double acc[4][4];   // launched with 256 threads: one 4 x 4 sub-tile each
    for (int a = 0; a < 4; ++a)
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] = 0.0;
    for (int k0 = j0; k0 < nd; k0 += 32) {
      for (int q = ex.tid; q < 32 * 64; q += ex.nt) {
        const int kk = q / 64, r = q % 64;
        const int k = k0 + kk, i = i0 + r, j = j0 + r;
        sA[q] = (k < nd && i < nd) ? pan[(int64_t)k * nf + nd + i] : 0.0;
        double xb = 0.0;
        if (k < nd && j < nd) xb = k == j ? 1.0 : (k > j ? pan[(int64_t)j * nf + k] : 0.0);
        sB[q] = xb;
      }
      ex.sync();
      for (int vt = ex.tid; vt < 256; vt += ex.nt) {
        const int tr = vt % 16, tc = vt / 16;
        double (*A)[4] = acc;
        for (int kk = 0; kk < 32; ++kk) {
          double li[4], rk[4];
          for (int a = 0; a < 4; ++a) li[a] = sA[kk * 64 + tr + 16 * a];
          for (int bb = 0; bb < 4; ++bb) rk[bb] = sB[kk * 64 + tc + 16 * bb];
          for (int a = 0; a < 4; ++a)
            for (int bb = 0; bb < 4; ++bb) A[a][bb] += li[a] * rk[bb];
        }
      }
      ex.sync();
    }
    for (int vt = ex.tid; vt < 256; vt += ex.nt) {
      const int tr = vt % 16, tc = vt / 16;
      double (*A)[4] = acc;
      for (int a = 0; a < 4; ++a)
        for (int bb = 0; bb < 4; ++bb) {
          const int i = i0 + tr + 16 * a, j = j0 + tc + 16 * bb;
          if (i < nd && j < nd) D[(int64_t)i * nd + j] = A[a][bb];   // D[j][i] = M[i][j]
        }
    }
  }
};

// Gauss-Jordan with partial pivoting on a row-major n x n matrix, one pivot
// column per pair of launches: (1) pivot search, row swap and scaling,
// (2) elimination of every other row, rows spread over many CTAs
struct KGJPivot {
  double* M;
  double* Inv;
  int64_t n, c;
  int* status;
  VB_HD void operator()(const KExec& ex, int) const {
    double* red = ex.smem;
    int* ired = reinterpret_cast<int*>(ex.smem + ex.nt);
    double best = -1.0;
    int bi = (int)c;
    for (int64_t r = c + ex.tid; r < n; r += ex.nt) {
      const double v = fabs(M[r * n + c]);
      if (v > best) { best = v; bi = (int)r; }
    }
    red[ex.tid] = best;
    ired[ex.tid] = bi;
    ex.sync();
    if (ex.tid == 0) {
      for (int t = 1; t < ex.nt; ++t)
        if (red[t] > red[0] || (red[t] == red[0] && ired[t] < ired[0])) { red[0] = red[t]; ired[0] = ired[t]; }
      if (!(red[0] > 0.0)) flag_error(status, 4);
    }
    ex.sync();
    const int64_t p = ired[0];
    if (p != c)
      for (int64_t j = ex.tid; j < n; j += ex.nt) {
        double t = M[c * n + j]; M[c * n + j] = M[p * n + j]; M[p * n + j] = t;
        t = Inv[c * n + j]; Inv[c * n + j] = Inv[p * n + j]; Inv[p * n + j] = t;
      }
    ex.sync();
    const double d = M[c * n + c] != 0.0 ? 1.0 / M[c * n + c] : 0.0;
    ex.sync();
    for (int64_t j = ex.tid; j < n; j += ex.nt) {
      if (j >= c) M[c * n + j] *= d;
      Inv[c * n + j] *= d;
    }
  }
};

struct KGJElim {
  double* M;
  double* Inv;
  int64_t n, c;
  int rows;
  VB_HD void operator()(const KExec& ex, int blk) const {
    for (int64_t r = (int64_t)blk * rows; r < (int64_t)(blk + 1) * rows && r < n; ++r) {
      if (r == c) continue;
      const double f = M[r * n + c];
      ex.sync();
      if (f != 0.0) {
        for (int64_t j = c + 1 + ex.tid; j < n; j += ex.nt) M[r * n + j] -= f * M[c * n + j];
        for (int64_t j = ex.tid; j < n; j += ex.nt) Inv[r * n + j] -= f * Inv[c * n + j];
      }
      ex.sync();
      if (ex.tid == 0) M[r * n + c] = 0.0;
    }
  }
};

// ----------------------------------------------------------------- apply

// c = H^T c and c = H c with the entity's reflectors, block-parallel
VB_HD inline void hh_T_par(const KExec& ex, const BddcView& V, const MacroDev& G, double* c, double* red) {
  if (G.hv_off < 0) return;
  for (int q = 0; q < G.r; ++q) {
    const double* h = V.hv + G.hv_off + (int64_t)q * G.n;
    double d = 0.0;
    for (int i = ex.tid; i < G.n; i += ex.nt) d += h[i] * c[i];
    d = block_sum(ex, d, red) * V.tau[G.tau_off + q];
    for (int i = ex.tid; i < G.n; i += ex.nt) c[i] -= d * h[i];
    ex.sync();
  }
}
VB_HD inline void hh_par(const KExec& ex, const BddcView& V, const MacroDev& G, double* c, double* red) {
  if (G.hv_off < 0) return;
  for (int q = G.r - 1; q >= 0; --q) {
    const double* h = V.hv + G.hv_off + (int64_t)q * G.n;
    double d = 0.0;
    for (int i = ex.tid; i < G.n; i += ex.nt) d += h[i] * c[i];
    d = block_sum(ex, d, red) * V.tau[G.tau_off + q];
    for (int i = ex.tid; i < G.n; i += ex.nt) c[i] -= d * h[i];
    ex.sync();
  }
}

// Coarse basis columns before the Neumann correction: entity g's primal
// coordinate q in sharing subdomain share[si] is the column H e_q of the
// entity's change of basis, scattered to the subdomain's local velocity
// DOFs (local column c0 + q); W is zero elsewhere (cleared beforehand).
struct CoarseWTask {
  int g, si, c0;
};
struct KCoarseW {
  BddcView V;
  const CoarseWTask* tasks;
  double* W;      // per subdomain: ncl columns, leading dimension nv + npress, at loc_off NC
  int2* wcols;    // per local row: the columns where W is nonzero (first, count)
  int NC;
  VB_HD void operator()(const KExec& ex, int t) const {
    const CoarseWTask T = tasks[t];
    const MacroDev G = V.macros[T.g];
    const SubDev S = V.subs[V.share[G.share_off + T.si]];
    const int nloc = S.nv + S.npress;
    const int* gi = V.gif + G.gif_off + (int64_t)T.si * G.n;
    double* c = ex.smem;
    double* red = ex.smem + G.n;
    for (int q = 0; q < G.r; ++q) {
      for (int a = ex.tid; a < G.n; a += ex.nt) c[a] = a == q ? 1.0 : 0.0;
      ex.sync();
      hh_par(ex, V, G, c, red);
      double* col = W + S.loc_off * NC + (int64_t)(T.c0 + q) * nloc;
      for (int a = ex.tid; a < G.n; a += ex.nt) col[V.iface[S.iface_off + gi[a]]] = c[a];
      ex.sync();
    }
    for (int a = ex.tid; a < G.n; a += ex.nt) wcols[S.loc_off + V.iface[S.iface_off + gi[a]]] = make_int2(T.c0, G.r);
  }
};
// the last local column: the subdomain's constant pressure p_0 = 1
struct KCoarseWP0 {
  BddcView V;
  double* W;
  int2* wcols;
  int NC;
  VB_HD void operator()(const KExec& ex, int i) const {
    const SubDev S = V.subs[i];
    const int nloc = S.nv + S.npress;
    double* col = W + S.loc_off * NC + (int64_t)(S.ncl - 1) * nloc + S.nv;
    for (int le = ex.tid; le < S.ne; le += ex.nt) {
      col[(int64_t)le * V.np] = 1.0;
      wcols[S.loc_off + S.nv + (int64_t)le * V.np] = make_int2(S.ncl - 1, 1);
    }
  }
};

// (1) r_G -> c = H^T r_G: primal part to the coarse rhs, dual part kept
struct KRestrict {
  BddcView V;
  const double* r;
  double* rC;
  double* dwork;
  double* part;
  VB_HD void operator()(const KExec& ex, int g) const {
    const MacroDev G = V.macros[g];
    double* c = ex.smem;
    double* red = ex.smem + G.n;
    double ss = 0.0;
    for (int a = ex.tid; a < G.n; a += ex.nt) {
      c[a] = r[V.mdofs[G.dofs_off + a]];
      ss += c[a] * c[a];
    }
    ss = block_sum(ex, ss, red);
    if (ex.tid == 0) part[g] = ss;
    hh_T_par(ex, V, G, c, red);
    for (int a = ex.tid; a < G.n; a += ex.nt) {
      if (a < G.r) rC[G.coarse0 + a] = c[a];
      else dwork[G.dual_off + a - G.r] = c[a];
    }
  }
};

// (2) subdomain constant-pressure residuals r_0,i
struct KRestrictP0 {
  BddcView V;
  const double* r;
  double* rC;
  double* part;
  int nmacro;
  VB_HD void operator()(const KExec& ex, int i) const {
    const SubDev S = V.subs[i];
    double s = 0.0;
    for (int le = ex.tid; le < S.ne; le += ex.nt) s += r[V.press[S.press_off + (int64_t)le * V.np]];
    s = block_sum(ex, s, ex.smem);
    if (ex.tid == 0) {
      rC[V.ncv + i] = s;
      part[nmacro + i] = s * s;
    }
  }
};

// deluxe GEMV tasks (DelTask): (face, first output index)

// out = D^T x on the dual coordinates of deluxe faces: one warp per output,
// lanes along the contiguous column of D (column-major storage)
struct KDeluxeT {
  BddcView V;
  const DelTask* tasks;
  const double* x;
  double* out;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const DelTask tk = tasks[blk];
    const MacroDev G = V.macros[tk.macro];
    const int nd = G.ndual;
    const double* xs = x + G.dual_off;
    double* xv = ex.smem;
    for (int i = ex.tid; i < nd; i += ex.nt) xv[i] = xs[i];
    ex.sync();
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    const int k1 = tk.k0 + 64 < nd ? tk.k0 + 64 : nd;
    for (int k = tk.k0 + w; k < k1; k += nw) {
      const double* Dk = V.deluxe + G.deluxe_off + (int64_t)k * nd;
      double a0 = 0.0, a1 = 0.0;
      int i = lane;
      for (; i + ws < nd; i += 2 * ws) { a0 += Dk[i] * xv[i]; a1 += Dk[i + ws] * xv[i + ws]; }
      if (i < nd) a0 += Dk[i] * xv[i];
      const double acc = warp_sum(a0 + a1);
      if (lane == 0) out[G.dual_off + k] = acc;
    }
  }
};

// avg = D (w0 - w1) + w1 on deluxe faces: one thread per output, rows of
// the column-major D read contiguously across threads
struct KDeluxeN {
  BddcView V;
  const DelTask* tasks;
  const double* w0;
  const double* w1;
  double* avg;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const DelTask tk = tasks[blk];
    const MacroDev G = V.macros[tk.macro];
    const int nd = G.ndual;
    double* dv = ex.smem;
    for (int i = ex.tid; i < nd; i += ex.nt) dv[i] = w0[G.dual_off + i] - w1[G.dual_off + i];
    ex.sync();
    const double* D = V.deluxe + G.deluxe_off;
    for (int k = tk.k0 + ex.tid; k < tk.k0 + 256 && k < nd; k += ex.nt) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int i = 0;
      for (; i + 3 < nd; i += 4) {
        a0 += D[(int64_t)i * nd + k] * dv[i];
        a1 += D[(int64_t)(i + 1) * nd + k] * dv[i + 1];
        a2 += D[(int64_t)(i + 2) * nd + k] * dv[i + 2];
        a3 += D[(int64_t)(i + 3) * nd + k] * dv[i + 3];
      }
      for (; i < nd; ++i) a0 += D[(int64_t)i * nd + k] * dv[i];
      avg[G.dual_off + k] = (a0 + a1) + (a2 + a3) + w1[G.dual_off + k];
    }
  }
};

// (3) scaled dual residual of each sharing subdomain, back to the original
// basis, written into its Neumann right-hand side (dt = D^T r on deluxe faces)
struct KScaleToNeumann {
  BddcView V;
  const double* dwork;
  const double* dt;
  double* XN;
  VB_HD void operator()(const KExec& ex, int g) const {
    const MacroDev G = V.macros[g];
    if (G.ndual == 0) return;
    double* c = ex.smem;
    double* red = ex.smem + G.n;
    const double* dr = dwork + G.dual_off;
    const double* dtr = dt + G.dual_off;
    for (int si = 0; si < G.nshare; ++si) {
      const int s = V.share[G.share_off + si];
      const SubDev S = V.subs[s];
      const ProbDev P = V.probs[S.neu];
      for (int a = ex.tid; a < G.n; a += ex.nt) {
        double v = 0.0;
        if (a >= G.r) {
          const int k = a - G.r;
          if (G.deluxe_off >= 0) {
            v = si == 0 ? dtr[k] : dr[k] - dtr[k];
          } else if (G.deluxe_e_off >= 0) {
            // deluxe edge: (D_s^T r)_k, column k of D_s
            const double* Dk = V.deluxe_e + G.deluxe_e_off + ((int64_t)si * G.ndual + k) * G.ndual;
            double acc = 0.0;
            for (int i = 0; i < G.ndual; ++i) acc += Dk[i] * dr[i];
            v = acc;
          } else {
            v = dr[k] / G.nshare;
          }
        }
        c[a] = v;
      }
      ex.sync();
      hh_par(ex, V, G, c, red);
      const int* gp = V.gpos + G.gpos_off + (int64_t)si * G.n;
      for (int a = ex.tid; a < G.n; a += ex.nt) XN[P.vec_off + gp[a]] = c[a];
      ex.sync();
    }
  }
};

// (4) local coarse rhs contributions Phi_Gamma^T g: one warp per coarse
// column, lanes along the interface rows; tasks of 8 columns
struct KCoarseLocal {
  BddcView V;
  const double* PG;
  const double* XN;
  double* cloc;
  int NC;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int nblk_per = (NC + 7) / 8;
    const int i = blk / nblk_per, c0 = (blk % nblk_per) * 8;
    const SubDev S = V.subs[i];
    const ProbDev P = V.probs[S.neu];
    const int* pv = V.pos_of_vdof + P.pv_off;
    const int ws = ex.nt >= 32 ? 32 : 1;
    const int nw = ex.nt / ws, w = ex.tid / ws, lane = ex.tid % ws;
    for (int c = c0 + w; c < c0 + 8 && c < S.ncl; c += nw) {
      const double* ph = PG + S.phi_off + (int64_t)c * S.niface;
      double acc = 0.0;
      for (int l = lane; l < S.niface; l += ws) {
        const int pos = pv[V.iface[S.iface_off + l]];
        if (pos >= 0) acc += ph[l] * XN[P.vec_off + pos];
      }
      acc = warp_sum(acc);
      if (lane == 0) cloc[(int64_t)i * NC + c] = acc;
    }
  }
};

struct KCoarseGather {
  BddcView V;
  const int* ptr;
  const int* sub;
  const int* loc;
  const double* cloc;
  double* rC;
  int NC;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < V.nc + 1 ? (int64_t)(blk + 1) * 256 : V.nc + 1;
    for (int64_t c = (int64_t)blk * 256 + ex.tid; c < hi; c += ex.nt) {
      if (c == V.nc) { rC[c] = 0.0; continue; }
      double acc = rC[c];
      for (int q = ptr[c]; q < ptr[c + 1]; ++q) acc += cloc[(int64_t)sub[q] * NC + loc[q]];
      rC[c] = acc;
    }
  }
};

// (6) u_C = K_C^{-1} r_C (bordered), one row per CTA
struct KCoarseSolve {
  const double* Kinv;
  const double* rC;
  double* uC;
  int64_t n;
  VB_HD void operator()(const KExec& ex, int row) const {
    const double* kr = Kinv + (int64_t)row * n;
    double acc = 0.0;
    for (int64_t j = ex.tid; j < n; j += ex.nt) acc += kr[j] * rC[j];
    acc = block_sum(ex, acc, ex.smem);
    if (ex.tid == 0) uC[row] = acc;
  }
};

// (8) w_Gamma = z_Gamma + Phi_Gamma u_C: tasks (subdomain, 256 interface rows)
struct KProlongLocal {
  BddcView V;
  const IfTask* tasks;
  const double* PG;
  const double* XN;
  const double* uC;
  double* wloc;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const IfTask tk = tasks[blk];
    const SubDev S = V.subs[tk.sub];
    const ProbDev P = V.probs[S.neu];
    const int* pv = V.pos_of_vdof + P.pv_off;
    const int64_t* g = V.coarse + S.coarse_off;
    double* uc = ex.smem;
    for (int c = ex.tid; c < S.ncl; c += ex.nt) uc[c] = uC[g[c]];
    ex.sync();
    for (int l = tk.l0 + ex.tid; l < tk.l0 + 256 && l < S.niface; l += ex.nt) {
      const int pos = pv[V.iface[S.iface_off + l]];
      double acc = pos >= 0 ? XN[P.vec_off + pos] : 0.0;
      for (int c = 0; c < S.ncl; ++c) acc += PG[S.phi_off + (int64_t)c * S.niface + l] * uc[c];
      wloc[S.iface_off + l] = acc;
    }
  }
};

// (9a) dual coordinates of each side's interface values: first side into
// w0, second into w1 (deluxe faces); the counting average into w0 otherwise
struct KAverageDual {
  BddcView V;
  const double* wloc;
  double* w0;
  double* w1;
  VB_HD void operator()(const KExec& ex, int g) const {
    const MacroDev G = V.macros[g];
    if (G.ndual == 0) return;
    double* w = ex.smem;
    double* red = ex.smem + G.n;
    for (int k = ex.tid; k < G.ndual; k += ex.nt) w0[G.dual_off + k] = 0.0;
    ex.sync();
    for (int si = 0; si < G.nshare; ++si) {
      const SubDev S = V.subs[V.share[G.share_off + si]];
      const int* gi = V.gif + G.gif_off + (int64_t)si * G.n;
      for (int a = ex.tid; a < G.n; a += ex.nt) w[a] = wloc[S.iface_off + gi[a]];
      ex.sync();
      hh_T_par(ex, V, G, w, red);
      if (G.deluxe_e_off >= 0) {
        // deluxe edge: w0 += D_s w_s (row k of D_s)
        ex.sync();
        const double* Ds = V.deluxe_e + G.deluxe_e_off + (int64_t)si * G.ndual * G.ndual;
        for (int k = ex.tid; k < G.ndual; k += ex.nt) {
          double acc = 0.0;
          for (int i = 0; i < G.ndual; ++i) acc += Ds[(int64_t)i * G.ndual + k] * w[G.r + i];
          w0[G.dual_off + k] += acc;
        }
      } else {
        for (int k = ex.tid; k < G.ndual; k += ex.nt) {
          const double v = w[G.r + k];
          if (G.deluxe_off >= 0) (si == 0 ? w0 : w1)[G.dual_off + k] = v;
          else w0[G.dual_off + k] += v / G.nshare;
        }
      }
      ex.sync();
    }
  }
};

// (9b) z_G = H [u_C primal; averaged dual] scattered to the system vector
struct KAverageOut {
  BddcView V;
  const double* avg_deluxe;
  const double* avg_count;
  const double* uC;
  double* z;
  VB_HD void operator()(const KExec& ex, int g) const {
    const MacroDev G = V.macros[g];
    double* c = ex.smem;
    double* red = ex.smem + G.n;
    const double* av = (G.deluxe_off >= 0 ? avg_deluxe : avg_count) + G.dual_off;
    for (int a = ex.tid; a < G.n; a += ex.nt) c[a] = a < G.r ? uC[G.coarse0 + a] : av[a - G.r];
    ex.sync();
    hh_par(ex, V, G, c, red);
    for (int a = ex.tid; a < G.n; a += ex.nt) z[V.mdofs[G.dofs_off + a]] = c[a];
  }
};

// (11) Dirichlet right-hand side: sgn * src at the problem positions, the
// pressure part projected onto sum-zero data
struct KDirRhs {
  BddcView V;
  const double* src;
  double sgn;
  double* XD;
  VB_HD void operator()(const KExec& ex, int i) const {
    const SubDev S = V.subs[i];
    const ProbDev P = V.probs[S.dir];
    double sg = 0.0;
    for (int le = ex.tid; le < S.ne; le += ex.nt) sg += sgn * src[V.press[S.press_off + (int64_t)le * V.np]];
    sg = block_sum(ex, sg, ex.smem);
    const double shift = sg / S.wsum;
    for (int pos = ex.tid; pos < P.n; pos += ex.nt) {
      const int dt = V.dtype[P.pos_off + pos], s2 = V.dsrc[P.pos_off + pos];
      double v = 0.0;
      if (dt == DT_VEL) v = sgn * src[V.vdof[S.vdof_off + s2]];
      else if (dt == DT_PRESS) v = sgn * src[V.press[S.press_off + s2]] - shift * V.wmean[S.press_off + s2];
      XD[P.vec_off + pos] = v;
    }
  }
};

// (13) interior velocity and pressure from the Dirichlet solution
struct KDirOut {
  BddcView V;
  const double* XD;
  const double* uC;   // may be null: no p_0 part
  double* z;
  VB_HD void operator()(const KExec& ex, int i) const {
    const SubDev S = V.subs[i];
    const ProbDev P = V.probs[S.dir];
    const int* pv = V.pos_of_vdof + P.pv_off;
    for (int v = ex.tid; v < S.nv; v += ex.nt) {
      const int pos = pv[v];
      if (pos >= 0) z[V.vdof[S.vdof_off + v]] = XD[P.vec_off + pos];
    }
    const int npk = V.np;
    double wp = 0.0;
    for (int q = ex.tid; q < S.npress; q += ex.nt) {
      const int le = q / npk, a = q % npk;
      const int e = V.sub_elems[S.elem_off + le];
      const int nK = (int)(V.offK[e + 1] - V.offK[e]);
      const int pos = V.elpos[P.elpos_off + V.elptr[P.elptr_off + le] + nK + a];
      wp += V.wmean[S.press_off + q] * (pos >= 0 ? XD[P.vec_off + pos] : 0.0);
    }
    wp = block_sum(ex, wp, ex.smem);
    const double m = wp / S.wsum;
    const double p0 = uC ? uC[V.ncv + i] : 0.0;
    for (int q = ex.tid; q < S.npress; q += ex.nt) {
      const int le = q / npk, a = q % npk;
      const int e = V.sub_elems[S.elem_off + le];
      const int nK = (int)(V.offK[e + 1] - V.offK[e]);
      const int pos = V.elpos[P.elpos_off + V.elptr[P.elptr_off + le] + nK + a];
      const double pz = pos >= 0 ? XD[P.vec_off + pos] : 0.0;
      z[V.press[S.press_off + q]] = pz + (a == 0 ? p0 - m : 0.0);
    }
  }
};

// ----------------------------------------------------------------- vectors
struct KDotPartial {
  const double* a;
  const double* b;
  int64_t n;
  double* part;
  VB_HD void operator()(const KExec& ex, int blk) const {
    double s = 0.0;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t lo = (int64_t)blk * chunk, hi = lo + chunk < n ? lo + chunk : n;
    for (int64_t i = lo + ex.tid; i < hi; i += ex.nt) s += a[i] * b[i];
    s = block_sum(ex, s, ex.smem);
    if (ex.tid == 0) part[blk] = s;
  }
};
struct KSumPartial {
  const double* part;
  int n;
  double* out;
  VB_HD void operator()(const KExec& ex, int) const {
    double s = 0.0;
    for (int i = ex.tid; i < n; i += ex.nt) s += part[i];
    s = block_sum(ex, s, ex.smem);
    if (ex.tid == 0) *out = s;
  }
};
struct KAxpby {   // y = a*x + b*y
  const double* x;
  double* y;
  double a, b;
  int64_t n;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < n ? (int64_t)(blk + 1) * 256 : n;
    for (int64_t i = (int64_t)blk * 256 + ex.tid; i < hi; i += ex.nt) y[i] = a * x[i] + b * y[i];
  }
};
struct KSub {     // r = f - Ax
  const double* f;
  const double* Ax;
  double* r;
  int64_t n;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < n ? (int64_t)(blk + 1) * 256 : n;
    for (int64_t i = (int64_t)blk * 256 + ex.tid; i < hi; i += ex.nt) r[i] = f[i] - Ax[i];
  }
};

}  // namespace vb

// =================================================================== host
namespace vb {

template <class T>
static void upload_vec(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
  if (h.empty()) { d.alloc(1); return; }
  d.upload(h, s);
}

static void build_batch(bddc* b, Batch& B, const std::vector<int>& probs, bool with_vectors) {
  B.probs = probs;
  int64_t vec = 0, uv = 0, nF = 0, nU = 0;
  // (height, -front cost, node): within a tree level the largest fronts come
  // first, so that the CTAs of the smallest ones fill the tail of the launch
  std::vector<std::tuple<int, double, int>> hn;
  B.maxnf = 1;
  B.maxh = 0;
  for (int q : probs) {
    ProbDev& P = b->h_probs[q];
    P.vec_off = vec;
    vec += P.n;
    const Problem& HP = b->H.probs[q];
    int base = (int)(&P - &b->h_probs[0]);
    (void)base;
    for (size_t k = 0; k < HP.nodes.size(); ++k) {
      int gid = b->h_probs[q].root - (int)HP.nodes.size() + 1 + (int)k;
      NodeDev& N = b->h_nodes[gid];
      // panels 4-element aligned with a leading dimension that is a
      // multiple of 4, so that 16-byte vector loads of columns are aligned
      N.ld = ((N.np + N.nb + 3) / 4) * 4;
      nF = ((nF + 3) / 4) * 4;
      N.panel_off = nF;
      nF += (int64_t)N.ld * N.np;
      N.upd_off = nU;
      nU += (int64_t)N.nb * N.nb;
      N.uvec_off = uv;
      uv += N.nb;
      const double nf = N.np + N.nb;
      hn.push_back({N.height, -(double)N.np * nf * nf, gid});
      B.maxh = std::max(B.maxh, N.height);
      B.maxnf = std::max(B.maxnf, N.np + N.nb);
    }
  }
  std::sort(hn.begin(), hn.end());
  B.level_ptr.assign(B.maxh + 2, 0);
  B.h_levels.clear();
  for (auto& pr : hn) {
    B.level_ptr[std::get<0>(pr) + 1]++;
    B.h_levels.push_back(std::get<2>(pr));
  }
  for (int h = 0; h <= B.maxh; ++h) B.level_ptr[h + 1] += B.level_ptr[h];
  // front-vector offsets and solve tasks per level
  if (b->h_fvoff.size() < b->h_nodes.size()) b->h_fvoff.resize(b->h_nodes.size(), 0);
  int64_t fv = 0;
  B.ptask_ptr.assign(B.maxh + 2, 0);
  B.btask_ptr.assign(B.maxh + 2, 0);
  B.fptask_ptr.assign(B.maxh + 2, 0);
  B.h_ptask.clear();
  B.h_btask.clear();
  B.h_fptask.clear();
  const int W = b->prec == 0 ? 2 : 4;   // rows per 16-byte vector load
  for (int h = 0; h <= B.maxh; ++h) {
    for (int q = B.level_ptr[h]; q < B.level_ptr[h + 1]; ++q) {
      const int t = B.h_levels[q];
      const NodeDev& N = b->h_nodes[t];
      b->h_fvoff[t] = fv;
      fv += N.np + N.nb;
      for (int s0 = 0; s0 < N.np; s0 += BCOLS) B.h_ptask.push_back({t, s0, std::min(BCOLS, N.np - s0)});
      const int nvp = (N.np + W - 1) / W;
      for (int s0 = 0; s0 < nvp; s0 += FVEC) B.h_fptask.push_back({t, s0, std::min(FVEC, nvp - s0)});
      const int a0 = (N.np / W) * W;
      const int nvb = N.nb > 0 ? (N.np + N.nb - a0 + W - 1) / W : 0;
      for (int s0 = 0; s0 < nvb; s0 += FVEC) B.h_btask.push_back({t, s0, std::min(FVEC, nvb - s0)});
    }
    B.ptask_ptr[h + 1] = (int)B.h_ptask.size();
    B.btask_ptr[h + 1] = (int)B.h_btask.size();
    B.fptask_ptr[h + 1] = (int)B.h_fptask.size();
  }
  B.nfv = fv;
  B.h_mtask.clear();
  B.h_etask.clear();
  for (int q : probs) {
    for (int s0 = 0; s0 < b->h_probs[q].n; s0 += TASK)
      B.h_mtask.push_back({q, s0, std::min(TASK, b->h_probs[q].n - s0)});
    for (int le = 0; le < (int)b->H.subs[b->H.probs[q].sub].elems.size(); ++le) B.h_etask.push_back({q, le});
  }
  // the element-share store spans every element of the mesh (each element
  // belongs to one subdomain, hence to one problem of the batch)
  B.ye_n = b->sys->h_eoff.back() + (int64_t)b->sys->dof.np * b->sys->topo.nE;
  B.vec_n = vec;
  B.uvec_n = uv;
  B.nF = nF;
  B.nU = nU;
  (void)with_vectors;
}

// factorization flops of a batch (partial LDL^T plus the L11 inversion);
// for deluxe problems without the skipped update blocks between two
// different entities at the root border
static double batch_gflop(bddc* b, const std::vector<int>& probs) {
  double f = 0;
  for (int q : probs) {
    const Problem& HP = b->H.probs[q];
    std::vector<double> cnt(HP.dl_macros.size());
    for (const Node& Nd : HP.nodes) {
      const double np = Nd.np, nf = Nd.np + Nd.nb;
      f += np * nf * nf - nf * np * np + np * np * np / 3.0 + np * np * np / 3.0;
      if (cnt.empty()) continue;
      std::fill(cnt.begin(), cnt.end(), 0.0);
      double tot = 0, diag = 0;
      for (int a = 0; a < Nd.nb; ++a) {
        const int g = HP.bgrp[HP.border[Nd.border_off + a]];
        if (g >= 0) { cnt[g] += 1; tot += 1; }
      }
      for (double c : cnt) diag += c * c;
      f -= np * (tot * tot - diag);
    }
  }
  return f * 1e-9;
}

static void upload_levels(bddc* b, Batch& B) {
  upload_vec(B.d_levels, B.h_levels, b->stream);
  upload_vec(B.d_ptask, B.h_ptask, b->stream);
  upload_vec(B.d_btask, B.h_btask, b->stream);
  upload_vec(B.d_fptask, B.h_fptask, b->stream);
  upload_vec(B.d_mtask, B.h_mtask, b->stream);
  upload_vec(B.d_etask, B.h_etask, b->stream);
}

template <class T>
static void factor_batch_t(bddc* b, Batch& B, const BddcView& V, DBuf<int>& status, DBuf<T>& Fs, DBuf<T>& Us) {
  Fs.alloc(std::max<int64_t>(B.nF, 1));
  Us.alloc(std::max<int64_t>(B.nU, 1));
  const size_t base = sizeof(double) * (std::max(2 * 64 * 32 + 128, B.maxnf) + 8);
  // diagnostics: with VEMBDDC_LEVEL_LOG set, every level's launch is timed
  // with CUDA events on the stream and printed to stderr
  static const bool level_log = std::getenv("VEMBDDC_LEVEL_LOG") != nullptr;
  // diagnostics: VEMBDDC_NO_SPLIT keeps every front of every level in one CTA
  static const bool split_off = std::getenv("VEMBDDC_NO_SPLIT") != nullptr;
  for (int h = 0; h <= B.maxh; ++h) {
    int cnt = B.level_ptr[h + 1] - B.level_ptr[h];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double lvl_flop = 0;
    if (level_log) {
      VB_CUDA(cudaEventCreate(&e0));
      VB_CUDA(cudaEventCreate(&e1));
      VB_CUDA(cudaEventRecord(e0, b->stream));
      for (int q = B.level_ptr[h]; q < B.level_ptr[h + 1]; ++q) {
        const NodeDev& Nd = b->h_nodes[B.h_levels[q]];
        const double np = Nd.np, nf = Nd.np + Nd.nb;
        lvl_flop += np * nf * nf - nf * np * np + 2.0 * np * np * np / 3.0;
      }
    }
    int nfmax = 0;
    for (int q = B.level_ptr[h]; q < B.level_ptr[h + 1]; ++q) {
      const NodeDev& Nd = b->h_nodes[B.h_levels[q]];
      nfmax = std::max(nfmax, Nd.np + Nd.nb);
    }
    // large fronts: 2 or 4 groups of 256 threads, each on its own trailing tile
    const int nthr = nfmax > 512 ? 1024 : (nfmax > 192 ? 512 : 256);
    const size_t gbase = sizeof(double) * (std::max((nthr / 256) * 2 * 64 * 32 + 128, B.maxnf) + 8);
    // FP32 fronts with trailing blocks beyond 64 rows: tensor-core updates
    if (std::is_same<T, float>::value && b->use_tc && nfmax > 96) {
      const size_t off = (base + 127) / 128 * 128;
      KFactor<float, true> f{V, B.d_levels.p + B.level_ptr[h], reinterpret_cast<float*>(Fs.p),
                             reinterpret_cast<float*>(Us.p), status.p, off};
      launch(f, cnt, 256, off + TC_SMEM_BYTES, b->stream);
    } else if (cnt <= 2 * 152 && nfmax >= 1024 && !split_off) {
      // few large fronts (the top of the trees): split form.  One CTA per
      // front assembles it, factors each outer panel and finally inverts
      // L11; the trailing update after each outer panel runs as one CTA
      // per 64 x 64 tile of every front, so that all SMs take part.
      KFactor<T> f{V, B.d_levels.p + B.level_ptr[h], Fs.p, Us.p, status.p};
      f.mode = 1;
      launch_mt<1024>(f, cnt, nthr, gbase, b->stream);
      int npmax = 0;
      for (int q = B.level_ptr[h]; q < B.level_ptr[h + 1]; ++q) npmax = std::max(npmax, b->h_nodes[B.h_levels[q]].np);
      constexpr int NBO = FrontSmem<T>::NBO;
      std::vector<FrontTile> tl;
      std::vector<int64_t> tptr(1, 0);
      for (int JB = 0; JB < npmax; JB += NBO) {
        for (int q = B.level_ptr[h]; q < B.level_ptr[h + 1]; ++q) {
          const int t = B.h_levels[q];
          const NodeDev& Nd = b->h_nodes[t];
          if (Nd.np <= JB) continue;
          const int JE = std::min(Nd.np, JB + NBO), nf = Nd.np + Nd.nb;
          const int nrt = (nf - JE + 63) / 64;
          for (int tk = 0; tk < nrt; ++tk)
            for (int ti = tk; ti < nrt; ++ti) tl.push_back({t, JE + 64 * ti, JE + 64 * tk});
        }
        tptr.push_back((int64_t)tl.size());
      }
      DBuf<FrontTile> dtl;
      upload_vec(dtl, tl, b->stream);
      const size_t tsm = sizeof(T) * (2 * 64 * 32 + NBO);
      for (int p = 0, JB = 0; JB < npmax; JB += NBO, ++p) {
        f.mode = 2;
        f.JB = JB;
        launch_mt<1024>(f, cnt, nthr, gbase, b->stream);
        launch(KFactorTiles<T>{V, dtl.p + tptr[p], Fs.p, Us.p, JB}, tptr[p + 1] - tptr[p], 256, tsm, b->stream);
      }
      f.mode = 3;
      launch_mt<1024>(f, cnt, nthr, gbase, b->stream);
      VB_CUDA(cudaStreamSynchronize(b->stream));   // the tile list is freed below
    } else {
      KFactor<T> f{V, B.d_levels.p + B.level_ptr[h], Fs.p, Us.p, status.p};
      launch_mt<1024>(f, cnt, nthr, gbase, b->stream);
    }
    if (level_log) {
      VB_CUDA(cudaEventRecord(e1, b->stream));
      VB_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      VB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      std::fprintf(stderr, "factor level %d: %d fronts, nf max %d, %.3f ms, %.1f Gflop (full fronts), %d threads\n", h,
                   cnt, nfmax, ms, lvl_flop * 1e-9, nthr);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
  }
}

static void factor_batch(bddc* b, Batch& B, const BddcView& V, DBuf<int>& status) {
  if (b->prec == 0) factor_batch_t<double>(b, B, V, status, B.F, B.U);
  else factor_batch_t<float>(b, B, V, status, B.F32, B.U32);
}

// captured graphs hold workspace addresses: drop them before a workspace
// is reallocated (they are captured again on next use; a graph being
// captured is not affected)
static void invalidate_graphs(bddc* b) {
  if (b->pcg_exec) { cudaGraphExecDestroy(b->pcg_exec); b->pcg_exec = nullptr; }
  if (b->app_exec) { cudaGraphExecDestroy(b->app_exec); b->app_exec = nullptr; }
}

template <class S, class D>
struct KCast {   // y = x converted, n entries
  const S* x;
  D* y;
  int64_t n;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t i = (int64_t)blk * ex.nt + ex.tid;
    if (i < n) y[i] = (D)x[i];
  }
};

// The sweep vectors are kept in the factor's precision T: for FP32 factors
// X is converted once on entry and once on exit, and the front and update
// vectors are FP32 views of their stores.
template <class T, int RB>
static void sweep_batch_rb(bddc* b, Batch& B, const BddcView& V, const T* Fp, double* Xd, double* UVd, int nrhs) {
  cudaStream_t st = b->stream;
  if (B.fv_nrhs < nrhs) {
    invalidate_graphs(b);
    B.FV.alloc(std::max<int64_t>(B.nfv * nrhs, 1));
    B.fv_nrhs = nrhs;
  }
  const int64_t nx = B.vec_n * nrhs;
  T* X = reinterpret_cast<T*>(Xd);
  T* UV = reinterpret_cast<T*>(UVd);
  T* FV = reinterpret_cast<T*>(B.FV.p);
  if constexpr (std::is_same<T, float>::value) {
    if ((int64_t)B.XF.n < nx) {
      invalidate_graphs(b);
      B.XF.alloc(std::max<int64_t>(nx, 1));
    }
    X = B.XF.p;
    launch(KCast<double, float>{Xd, X, nx}, (nx + 255) / 256, 256, 0, st);
  }
  const size_t sm = sizeof(T) * (RB * (B.maxnf + 8));
  const size_t smf = sm + sizeof(double) * FWARPS * FVEC * 4 * RB;   // + partial sums of the warps
  VB_CHECK(smf <= 227 * 1024, VEM_EINVAL, "front too large for the sweep kernels' shared memory");
  const int64_t* fvo = b->d_fvoff.p;
  for (int h = 0; h <= B.maxh; ++h) {
    const int cnt = B.level_ptr[h + 1] - B.level_ptr[h];
    const int fp_t = B.fptask_ptr[h + 1] - B.fptask_ptr[h];
    const int nb_t = B.btask_ptr[h + 1] - B.btask_ptr[h];
    launch(KFwdGather<T>{V, B.d_levels.p + B.level_ptr[h], X, UV, FV, fvo, nrhs}, cnt, 128, 0, st);
    // FP32, single right-hand side: registers capped for 6 (forward) or 5
    // (backward) resident CTAs per SM
    // (these kernels wait on memory; occupancy hides the latency)
    if constexpr (RB == 1 && std::is_same<T, float>::value) {
      launch_lb<6>(KFwdPivots<T, RB>{V, B.d_fptask.p + B.fptask_ptr[h], Fp, FV, fvo, X, nrhs}, fp_t, smf, st);
      launch_lb<6>(KFwdBorder<T, RB>{V, B.d_btask.p + B.btask_ptr[h], Fp, FV, fvo, X, UV, nrhs}, nb_t, smf, st);
    } else {
      launch(KFwdPivots<T, RB>{V, B.d_fptask.p + B.fptask_ptr[h], Fp, FV, fvo, X, nrhs}, fp_t, 32 * FWARPS, smf,
             st);
      launch(KFwdBorder<T, RB>{V, B.d_btask.p + B.btask_ptr[h], Fp, FV, fvo, X, UV, nrhs}, nb_t, 32 * FWARPS,
             smf, st);
    }
  }
  for (int h = B.maxh; h >= 0; --h) {
    const int np_t = B.ptask_ptr[h + 1] - B.ptask_ptr[h];
    if constexpr (RB == 1 && std::is_same<T, float>::value) {
      launch_lb<5>(KBwdBorder<T, RB>{V, B.d_ptask.p + B.ptask_ptr[h], Fp, X, FV, fvo, nrhs}, np_t, sm, st);
      launch_lb<5>(KBwdPivots<T, RB>{V, B.d_ptask.p + B.ptask_ptr[h], Fp, FV, fvo, X, nrhs}, np_t, sm, st);
    } else {
      launch(KBwdBorder<T, RB>{V, B.d_ptask.p + B.ptask_ptr[h], Fp, X, FV, fvo, nrhs}, np_t, 256, sm, st);
      launch(KBwdPivots<T, RB>{V, B.d_ptask.p + B.ptask_ptr[h], Fp, FV, fvo, X, nrhs}, np_t, 256, sm, st);
    }
  }
  if constexpr (std::is_same<T, float>::value) launch(KCast<float, double>{X, Xd, nx}, (nx + 255) / 256, 256, 0, st);
}

template <class T>
static void sweep_batch(bddc* b, Batch& B, const BddcView& V, const T* Fp, double* X, double* UV, int nrhs) {
  if (nrhs >= 4) sweep_batch_rb<T, 4>(b, B, V, Fp, X, UV, nrhs);
  else sweep_batch_rb<T, 1>(b, B, V, Fp, X, UV, nrhs);
}

struct KAxpyN {   // y += x over n entries
  const double* x;
  double* y;
  int64_t n;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < n ? (int64_t)(blk + 1) * 256 : n;
    for (int64_t i = (int64_t)blk * 256 + ex.tid; i < hi; i += ex.nt) y[i] += x[i];
  }
};

// local solves of a batch, X (right-hand sides) overwritten by the
// solutions; FP32-local factors get one step of refinement with the
// residual computed in FP64 from the element matrices
static void solve_batch(bddc* b, Batch& B, const BddcView& V, double* X, double* UV, int nrhs) {
  if (b->prec == 0) {
    sweep_batch<double>(b, B, V, B.F.p, X, UV, nrhs);
    return;
  }
  if (b->prec == 2) {
    sweep_batch<float>(b, B, V, B.F32.p, X, UV, nrhs);
    return;
  }
  cudaStream_t st = b->stream;
  const int64_t n = B.vec_n * nrhs;
  if ((int64_t)B.XB.n < n) {
    invalidate_graphs(b);
    B.XB.alloc(std::max<int64_t>(n, 1));
    B.XR.alloc(std::max<int64_t>(n, 1));
  }
  VB_CUDA(cudaMemcpyAsync(B.XB.p, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  sweep_batch<float>(b, B, V, B.F32.p, X, UV, nrhs);
  const int chunk = std::min(nrhs, 16);
  if ((int64_t)B.YE.n < B.ye_n * chunk) {
    invalidate_graphs(b);
    B.YE.alloc(B.ye_n * chunk);
  }
  const size_t esm = sizeof(double) * 4 * (b->sys->nKmax + b->sys->dof.np);
  for (int it = 0; it < b->refine; ++it) {
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
      const int nr = std::min(chunk, nrhs - r0);
      const int64_t ne = (int64_t)B.h_etask.size();
      if (V.A2 && nr >= 4)
        launch(KElemProduct<4, true>{V, B.d_etask.p, X, B.YE.p, nrhs, r0, nr}, ne, 128, 2 * esm, st);
      else if (V.A2)
        launch(KElemProduct<1, true>{V, B.d_etask.p, X, B.YE.p, nrhs, r0, nr}, ne, 128, 2 * esm, st);
      else if (nr >= 4)
        launch(KElemProduct<4>{V, B.d_etask.p, X, B.YE.p, nrhs, r0, nr}, ne, 128, esm, st);
      else
        launch(KElemProduct<1>{V, B.d_etask.p, X, B.YE.p, nrhs, r0, nr}, ne, 128, esm, st);
      launch(KGatherResidual{V, B.d_mtask.p, B.XB.p, X, B.YE.p, B.XR.p, b->d_mcon_ptr.p, b->d_mcon_vdof.p,
                             b->d_mcon_coef.p, nrhs, r0, nr}, (int64_t)B.h_mtask.size(), 128, 0, st);
    }
    sweep_batch<float>(b, B, V, B.F32.p, B.XR.p, UV, nrhs);
    launch(KAxpyN{B.XR.p, X, n}, (n + 255) / 256, 256, 0, st);
  }
}

static int max_macro_n(bddc* b) {
  int m = 1;
  for (auto& G : b->h_macros) m = std::max(m, G.n);
  return m;
}

// z = M^{-1} r (BDDC with the Dirichlet harmonic extension), system layout
static void apply_bddc(bddc* b, const double* r, double* z) {
  vem_system* s = b->sys;
  const BddcView V = make_view(b);
  cudaStream_t st = b->stream;
  const int nmac = (int)b->h_macros.size();
  const int N = b->H.N;
  const size_t msm = sizeof(double) * (3 * max_macro_n(b) + 256 + 8);
  const size_t dsm = sizeof(double) * (b->max_nd + 8);
  const int NC = b->NC;
  b->XN.zero(st);
  launch(KRestrict{V, r, b->rC.p, b->dwork.p, b->part.p}, nmac, 256, msm, st);
  launch(KRestrictP0{V, r, b->rC.p, b->part.p, nmac}, N, 256, sizeof(double) * 256, st);
  launch(KDeluxeT{V, b->d_dtT.p, b->dwork.p, b->dtw.p}, (int64_t)b->h_dtT.size(), 256, dsm, st);
  launch(KScaleToNeumann{V, b->dwork.p, b->dtw.p, b->XN.p}, nmac, 256, msm, st);
  launch(KCoarseLocal{V, b->d_phi.p, b->XN.p, b->cloc.p, NC}, (int64_t)N * ((NC + 7) / 8), 256, 0, st);
  launch(KCoarseGather{V, b->d_cg_ptr.p, b->d_cg_sub.p, b->d_cg_loc.p, b->cloc.p, b->rC.p, NC},
         (b->nc + 1 + 255) / 256, 256, 0, st);
  launch(KCoarseSolve{b->d_Kinv.p, b->rC.p, b->uC.p, b->nc + 1}, b->nc + 1, 256, sizeof(double) * 256, st);
  solve_batch(b, b->bn, V, b->XN.p, b->UVN.p, 1);
  launch(KProlongLocal{V, b->d_ift.p, b->d_phi.p, b->XN.p, b->uC.p, b->wloc.p}, (int64_t)b->h_ift.size(), 256,
         sizeof(double) * (NC + 8), st);
  launch(KAverageDual{V, b->wloc.p, b->dwork.p, b->wd1.p}, nmac, 256, msm, st);
  launch(KDeluxeN{V, b->d_dtN.p, b->dwork.p, b->wd1.p, b->avgd.p}, (int64_t)b->h_dtN.size(), 256, dsm, st);
  VB_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * s->n, st));
  launch(KAverageOut{V, b->avgd.p, b->dwork.p, b->uC.p, z}, nmac, 256, msm, st);
  spmv(s, z, b->y.p, st);
  launch(KDirRhs{V, b->y.p, -1.0, b->XD.p}, N, 256, sizeof(double) * 256, st);
  solve_batch(b, b->bd, V, b->XD.p, b->UVD.p, 1);
  launch(KDirOut{V, b->XD.p, b->uC.p, z}, N, 256, sizeof(double) * 256, st);
}

static double dot(bddc* b, const double* x, const double* y, int64_t n) {
  launch(KDotPartial{x, y, n, b->part.p + b->part.n - 1024 - 1}, 1024, 256, sizeof(double) * 256, b->stream);
  launch(KSumPartial{b->part.p + b->part.n - 1024 - 1, 1024, b->scal.p}, 1, 256, sizeof(double) * 256, b->stream);
  double h;
  VB_CUDA(cudaMemcpyAsync(&h, b->scal.p, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  VB_CUDA(cudaStreamSynchronize(b->stream));
  return h;
}

static double iface_norm(bddc* b, const double* r) {
  const BddcView V = make_view(b);
  const int nmac = (int)b->h_macros.size();
  const size_t msm = sizeof(double) * (3 * max_macro_n(b) + 256 + 8);
  launch(KRestrict{V, r, b->rC.p, b->dwork.p, b->part.p}, nmac, 256, msm, b->stream);
  launch(KRestrictP0{V, r, b->rC.p, b->part.p, nmac}, b->H.N, 256, sizeof(double) * 256, b->stream);
  launch(KSumPartial{b->part.p, nmac + b->H.N, b->scal.p}, 1, 256, sizeof(double) * 256, b->stream);
  double h;
  VB_CUDA(cudaMemcpyAsync(&h, b->scal.p, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  VB_CUDA(cudaStreamSynchronize(b->stream));
  return std::sqrt(h);
}

static void lanczos(const std::vector<double>& al, const std::vector<double>& be, double& lmin, double& lmax) {
  const int m = (int)al.size();
  if (m == 0) { lmin = lmax = 1.0; return; }
  std::vector<double> d(m), e(m, 0.0);
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j < m - 1) e[j] = std::sqrt(be[j]) / al[j];
  }
  // Gershgorin bounds, then bisection with Sturm counts
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < m; ++j) {
    double rr = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j < m - 1 ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - rr);
    hi = std::max(hi, d[j] + rr);
  }
  auto count = [&](double x) {   // eigenvalues < x
    int c = 0;
    double q = d[0] - x;
    if (q < 0) c++;
    for (int j = 1; j < m; ++j) {
      if (q == 0.0) q = 1e-300;
      q = d[j] - x - e[j - 1] * e[j - 1] / q;
      if (q < 0) c++;
    }
    return c;
  };
  auto kth = [&](int k) {
    double a = lo, bb = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + bb);
      if (count(mid) > k) bb = mid; else a = mid;
    }
    return 0.5 * (a + bb);
  };
  lmin = kth(0);
  lmax = kth(m - 1);
}

// ------------------------------------------------------- graph-captured PCG
// Device scalars of the PCG loop
enum { PS_RZ = 0, PS_RZN, PS_PAP, PS_ALPHA, PS_BETA, PS_NR2, PS_TOL, PS_IT, PS_MAXIT, PS_STATUS, PS_COUNT };
// PS_STATUS: 0 running, 1 converged, 2 breakdown, 3 maxit reached

// beta_{j-1} = (r_j, z_j) / (r_{j-1}, z_{j-1}) (0 at j = 0), recorded for Lanczos
struct KPcgBeta {
  double* s;
  double* be;
  __device__ void operator()(const KExec& ex, int) const {
    if (ex.tid != 0) return;
    const int it = (int)s[PS_IT];
    const double rzn = s[PS_RZN];
    double beta = 0.0;
    if (it > 0) {
      beta = rzn / s[PS_RZ];
      be[it - 1] = beta;
    }
    s[PS_BETA] = beta;
    s[PS_RZ] = rzn;
  }
};
// p = z + beta p
struct KPcgDirection {
  const double* z;
  double* p;
  const double* s;
  int64_t n;
  __device__ void operator()(const KExec& ex, int blk) const {
    const double beta = s[PS_BETA];
    const int64_t hi = (int64_t)(blk + 1) * 256 < n ? (int64_t)(blk + 1) * 256 : n;
    for (int64_t i = (int64_t)blk * 256 + ex.tid; i < hi; i += ex.nt) p[i] = z[i] + beta * p[i];
  }
};
// alpha = (r, z) / (p, K p), or breakdown when p^T K p <= 0 or non-finite
struct KPcgAlpha {
  double* s;
  double* al;
  __device__ void operator()(const KExec& ex, int) const {
    if (ex.tid != 0) return;
    const double pAp = s[PS_PAP], rz = s[PS_RZ];
    if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(rz)) {
      s[PS_STATUS] = 2.0;
      s[PS_ALPHA] = 0.0;
      return;
    }
    const double alpha = rz / pAp;
    s[PS_ALPHA] = alpha;
    al[(int)s[PS_IT]] = alpha;
  }
};
// x += alpha p, r -= alpha K p (skipped after a breakdown)
struct KPcgUpdate {
  const double* p;
  const double* Ap;
  double* x;
  double* r;
  const double* s;
  int64_t n;
  __device__ void operator()(const KExec& ex, int blk) const {
    if (s[PS_STATUS] != 0.0) return;
    const double alpha = s[PS_ALPHA];
    const int64_t hi = (int64_t)(blk + 1) * 256 < n ? (int64_t)(blk + 1) * 256 : n;
    for (int64_t i = (int64_t)blk * 256 + ex.tid; i < hi; i += ex.nt) {
      x[i] = alpha * p[i] + x[i];
      r[i] = -alpha * Ap[i] + r[i];
    }
  }
};
// iteration count, stop rule ||r_Gamma|| <= rtol ||r_Gamma,0|| (tolerance
// pre-multiplied), maxit; sets the loop condition
struct KPcgCheck {
  double* s;
  cudaGraphConditionalHandle h;
  __device__ void operator()(const KExec& ex, int) const {
    if (ex.tid != 0) return;
    unsigned int more = 0;
    if (s[PS_STATUS] == 0.0) {
      const double it = s[PS_IT] + 1.0;
      s[PS_IT] = it;
      if (sqrt(s[PS_NR2]) <= s[PS_TOL]) s[PS_STATUS] = 1.0;
      else if (it >= s[PS_MAXIT]) s[PS_STATUS] = 3.0;
      else more = 1;
    }
    cudaGraphSetConditional(h, more);
  }
};

static cudaStream_t capture_stream(bddc* b) {
  if (!b->cap_stream) VB_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  return b->cap_stream;
}

// (a, b) -> s[slot], deterministic two-pass sum
static void dot_to(bddc* b, const double* x, const double* y, int64_t n, double* out) {
  launch(KDotPartial{x, y, n, b->part.p + b->part.n - 1024 - 1}, 1024, 256, sizeof(double) * 256, b->stream);
  launch(KSumPartial{b->part.p + b->part.n - 1024 - 1, 1024, out}, 1, 256, sizeof(double) * 256, b->stream);
}

// ||r_Gamma||^2 (interface velocity and p_0 parts) -> out
static void iface_norm2_to(bddc* b, const double* r, double* out) {
  const BddcView V = make_view(b);
  const int nmac = (int)b->h_macros.size();
  const size_t msm = sizeof(double) * (3 * max_macro_n(b) + 256 + 8);
  launch(KRestrict{V, r, b->rC.p, b->dwork.p, b->part.p}, nmac, 256, msm, b->stream);
  launch(KRestrictP0{V, r, b->rC.p, b->part.p, nmac}, b->H.N, 256, sizeof(double) * 256, b->stream);
  launch(KSumPartial{b->part.p, nmac + b->H.N, out}, 1, 256, sizeof(double) * 256, b->stream);
}

// one PCG iteration on (x, r, p) with the device scalars; same operations
// and order as the host-driven loop
static void pcg_body(bddc* b, cudaGraphConditionalHandle h) {
  const int64_t n = b->sys->n;
  const int nblk = (int)((n + 255) / 256);
  double* s = b->pcg_s.p;
  apply_bddc(b, b->r.p, b->z.p);
  dot_to(b, b->r.p, b->z.p, n, s + PS_RZN);
  launch(KPcgBeta{s, b->pcg_be.p}, 1, 32, 0, b->stream);
  launch(KPcgDirection{b->z.p, b->p.p, s, n}, nblk, 256, 0, b->stream);
  spmv(b->sys, b->p.p, b->Ap.p, b->stream);
  dot_to(b, b->p.p, b->Ap.p, n, s + PS_PAP);
  launch(KPcgAlpha{s, b->pcg_al.p}, 1, 32, 0, b->stream);
  launch(KPcgUpdate{b->p.p, b->Ap.p, b->xg.p, b->r.p, s, n}, nblk, 256, 0, b->stream);
  iface_norm2_to(b, b->r.p, s + PS_NR2);
  launch(KPcgCheck{s, h}, 1, 32, 0, b->stream);
}

// Captures the PCG loop: a graph with one conditional while node whose body
// is pcg_body (the condition starts at 1 on every launch)
static void pcg_capture(bddc* b) {
  if (b->pcg_exec) { VB_CUDA(cudaGraphExecDestroy(b->pcg_exec)); b->pcg_exec = nullptr; }
  cudaGraph_t g = nullptr;
  VB_CUDA(cudaGraphCreate(&g, 0));
  cudaStream_t cs = capture_stream(b);
  cudaStream_t saved = b->stream;
  try {
    cudaGraphConditionalHandle h;
    VB_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VB_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int64_t l0 = g_launches.load();
    VB_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    b->stream = cs;
    try {
      pcg_body(b, h);
    } catch (...) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(cs, &tmp);
      (void)cudaGetLastError();
      throw;
    }
    b->stream = saved;
    VB_CUDA(cudaStreamEndCapture(cs, &body));
    b->pcg_body_launches = g_launches.load() - l0;
    g_launches.fetch_sub(b->pcg_body_launches);   // counted when the graph runs
    VB_CUDA(cudaGraphInstantiate(&b->pcg_exec, g, 0));
  } catch (...) {
    b->stream = saved;
    cudaGraphDestroy(g);
    throw;
  }
  cudaGraphDestroy(g);
}

// z = M^{-1} r through a captured graph (re-captured when r or z change)
static void apply_graph(bddc* b, const double* r, double* z) {
  if (!b->app_exec || b->app_r != r || b->app_z != z) {
    if (b->app_exec) { VB_CUDA(cudaGraphExecDestroy(b->app_exec)); b->app_exec = nullptr; }
    cudaStream_t cs = capture_stream(b);
    cudaStream_t saved = b->stream;
    cudaGraph_t g = nullptr;
    const int64_t l0 = g_launches.load();
    VB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    b->stream = cs;
    try {
      apply_bddc(b, r, z);
    } catch (...) {
      b->stream = saved;
      cudaStreamEndCapture(cs, &g);
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      throw;
    }
    b->stream = saved;
    VB_CUDA(cudaStreamEndCapture(cs, &g));
    b->app_launches = g_launches.load() - l0;
    g_launches.fetch_sub(b->app_launches);
    cudaError_t e = cudaGraphInstantiate(&b->app_exec, g, 0);
    cudaGraphDestroy(g);
    VB_CUDA(e);
    b->app_r = r;
    b->app_z = z;
  }
  VB_CUDA(cudaGraphLaunch(b->app_exec, b->stream));
  g_launches.fetch_add(b->app_launches);
}

// ------------------------------------------------ adaptive coarse space (S7)
// Sec. 6.  For every macro face F with sides i, j and dual coordinates F_D:
//   S~_s = (E^T K_rr^(s)-1 E)^-1 = M_s^-1 (E: the dual basis columns H e_c,
//   K_rr the constrained Neumann matrix), so A = S~_i : S~_j = (M_i + M_j)^-1;
//   B = S_i : S_j = S_j (S_i + S_j)^-1 S_i = S_j D_i (D_i the deluxe block).
// A psi = lambda B psi is solved as G^T B G y = mu y with M_i + M_j = G G^T,
// psi = G y and lambda = 1/mu; eigenvalues lambda < 1/theta (mu > theta) give
// the new primal functionals B psi on F_D, which are mapped back to the
// face's DOFs with H.  The eigenvector scaling differs from a B-normalised
// one by a factor per vector, which leaves the primal space unchanged.
struct AdaptTask {
  int sub, macro, si, c0, ncol;
  int64_t moff;
};

// column c of a task: H e_{r+c0+c} on the macro's DOFs, written at their
// positions in the subdomain's Neumann problem (the rest of X is zero)
struct KAdaptRhs {
  BddcView V;
  const AdaptTask* tasks;
  double* X;
  int nrhs;
  __device__ void operator()(const KExec& ex, int blk) const {
    const AdaptTask tk = tasks[blk / nrhs];
    const int c = blk % nrhs;
    if (c >= tk.ncol) return;
    const MacroDev G = V.macros[tk.macro];
    const ProbDev P = V.probs[V.subs[tk.sub].neu];
    double* v = ex.smem;
    double* red = ex.smem + G.n;
    for (int a = ex.tid; a < G.n; a += ex.nt) v[a] = a == G.r + tk.c0 + c ? 1.0 : 0.0;
    ex.sync();
    hh_par(ex, V, G, v, red);
    const int* gp = V.gpos + G.gpos_off + (int64_t)tk.si * G.n;
    for (int a = ex.tid; a < G.n; a += ex.nt) X[P.vec_off * nrhs + (int64_t)c * P.n + gp[a]] = v[a];
  }
};

// column c0+c of M_s: the dual coordinates (H^T x)[r:] of the solution
struct KAdaptGather {
  BddcView V;
  const AdaptTask* tasks;
  const double* X;
  double* M;
  int nrhs;
  __device__ void operator()(const KExec& ex, int blk) const {
    const AdaptTask tk = tasks[blk / nrhs];
    const int c = blk % nrhs;
    if (c >= tk.ncol) return;
    const MacroDev G = V.macros[tk.macro];
    const ProbDev P = V.probs[V.subs[tk.sub].neu];
    double* v = ex.smem;
    double* red = ex.smem + G.n;
    const int* gp = V.gpos + G.gpos_off + (int64_t)tk.si * G.n;
    for (int a = ex.tid; a < G.n; a += ex.nt) v[a] = X[P.vec_off * nrhs + (int64_t)c * P.n + gp[a]];
    ex.sync();
    hh_T_par(ex, V, G, v, red);
    const int nd = G.n - G.r;
    for (int k = ex.tid; k < nd; k += ex.nt) M[tk.moff + (int64_t)(tk.c0 + c) * nd + k] = v[G.r + k];
  }
};

// N = M_i + M_j per face (items: a = M_i, b = M_j, c = N offsets)
struct KAddPair {
  const double* M;
  double* Nout;
  const DenseItem* items;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int64_t nn = (int64_t)it.n * it.n;
    for (int64_t q = ex.tid; q < nn; q += ex.nt) Nout[it.c + q] = M[it.a + q] + M[it.b + q];
  }
};

// Adaptive primal rows of every macro face (in the face's DOF order, one
// functional of length n per row) into extra[macro]; returns the count
static int adaptive_rows(bddc* b, std::vector<std::vector<double>>& extra) {
  cudaStream_t st = b->stream;
  const BddcView V = make_view(b);
  const int nfc = (int)b->sf_faces.size();
  extra.assign(b->h_macros.size(), {});
  if (nfc == 0) return 0;
  const int N = b->H.N;
  constexpr int MAXSEL = 64;
  std::vector<int> nd(nfc);
  std::vector<int64_t> mi(nfc), mj(nfc), fo(nfc), yo(nfc);
  int64_t mtot = 0, ftot = 0, ytot = 0;
  int nmax = 1;
  for (int t = 0; t < nfc; ++t) {
    nd[t] = b->h_macros[b->sf_faces[t]].ndual;
    const int64_t q = (int64_t)nd[t] * nd[t];
    mi[t] = mtot;
    mj[t] = mtot + q;
    mtot += 2 * q;
    fo[t] = ftot;
    ftot += q;
    yo[t] = ytot;
    ytot += (int64_t)MAXSEL * nd[t];
    nmax = std::max(nmax, b->h_macros[b->sf_faces[t]].n);
  }
  // ---- M_s = E^T K_rr^-1 E: multi-RHS Neumann solves, one face per
  // subdomain at a time ("slots"), NCc dual columns per solve
  DBuf<double> M(std::max<int64_t>(mtot, 1));
  std::vector<std::vector<std::pair<int, int>>> sub_faces(N);
  for (int t = 0; t < nfc; ++t) {
    const Macro& G = b->H.macros[b->sf_faces[t]];
    sub_faces[G.share[0]].push_back({t, 0});
    sub_faces[G.share[1]].push_back({t, 1});
  }
  size_t nslot = 0;
  for (auto& v : sub_faces) nslot = std::max(nslot, v.size());
  constexpr int NCc = 32;
  DBuf<double> X(std::max<int64_t>(b->bn.vec_n * NCc, 1)), UV(std::max<int64_t>(b->bn.uvec_n * NCc, 1));
  DBuf<AdaptTask> dtasks;
  const size_t asm_ = sizeof(double) * (nmax + 256);
  for (size_t slot = 0; slot < nslot; ++slot) {
    int maxnd = 0;
    for (int i = 0; i < N; ++i)
      if (slot < sub_faces[i].size()) maxnd = std::max(maxnd, nd[sub_faces[i][slot].first]);
    for (int c0 = 0; c0 < maxnd; c0 += NCc) {
      std::vector<AdaptTask> tasks;
      for (int i = 0; i < N; ++i) {
        if (slot >= sub_faces[i].size()) continue;
        const auto [t, si] = sub_faces[i][slot];
        if (c0 >= nd[t]) continue;
        tasks.push_back({i, b->sf_faces[t], si, c0, std::min(NCc, nd[t] - c0), si == 0 ? mi[t] : mj[t]});
      }
      if (tasks.empty()) continue;
      upload_vec(dtasks, tasks, st);
      X.zero(st);
      launch(KAdaptRhs{V, dtasks.p, X.p, NCc}, (int64_t)tasks.size() * NCc, 256, asm_, st);
      solve_batch(b, b->bn, V, X.p, UV.p, NCc);
      launch(KAdaptGather{V, dtasks.p, X.p, M.p, NCc}, (int64_t)tasks.size() * NCc, 256, asm_, st);
    }
  }
  // ---- dense per-face steps
  std::vector<DenseItem> it_add(nfc), it_b(nfc), it_f(nfc), it_t1(nfc), it_c(nfc), it_tri(nfc), it_rows(nfc);
  std::vector<GemmTask> gt;
  for (int t = 0; t < nfc; ++t) {
    const MacroDev& G = b->h_macros[b->sf_faces[t]];
    it_add[t] = {nd[t], mi[t], mj[t], fo[t]};                 // Nf = M_i + M_j
    it_b[t] = {nd[t], b->sf_j[t], G.deluxe_off, fo[t]};       // Bf = S_j D_i
    it_f[t] = {nd[t], fo[t], 0, 0};                           // in-place on one matrix
    it_t1[t] = {nd[t], fo[t], fo[t], fo[t]};                  // T1 = Bf G ; Cf = G^T T1
    it_tri[t] = {nd[t], fo[t], 2 * fo[t], fo[t]};             // Cf ; d/e (2n per face) ; tau
    it_rows[t] = {nd[t], fo[t], fo[t], 0};                    // G (in Nf) ; Bf
    const int ntl = (nd[t] + 63) / 64;
    for (int ti = 0; ti < ntl; ++ti)
      for (int tj = 0; tj < ntl; ++tj) gt.push_back({t, ti, tj});
  }
  DBuf<DenseItem> d_add, d_b, d_f, d_t1, d_tri, d_rows;
  DBuf<GemmTask> d_gt;
  upload_vec(d_add, it_add, st);
  upload_vec(d_b, it_b, st);
  upload_vec(d_f, it_f, st);
  upload_vec(d_t1, it_t1, st);
  upload_vec(d_tri, it_tri, st);
  upload_vec(d_rows, it_rows, st);
  upload_vec(d_gt, gt, st);
  const int64_t ft = std::max<int64_t>(ftot, 1);
  DBuf<double> Nf(ft), Bf(ft), T1(ft), Cf(ft), DE(2 * ft), TAU(ft), Y(std::max<int64_t>(ytot, 1)),
      LAM((int64_t)nfc * MAXSEL);
  DBuf<int> cnt(nfc), status(1);
  status.zero(st);
  const size_t gsm = sizeof(double) * 2 * 16 * 65;
  launch(KAddPair{M.p, Nf.p, d_add.p}, nfc, 256, 0, st);
  launch(KSymmetrize{Nf.p, d_f.p}, nfc, 256, 0, st);
  launch(KBatchGemm{b->d_sf.p, b->d_deluxe.p, Bf.p, d_b.p, d_gt.p, 0, 1.0, 0.0}, (int64_t)gt.size(), 256, gsm, st);
  launch(KSymmetrize{Bf.p, d_f.p}, nfc, 256, 0, st);
  launch(KCholesky{Nf.p, d_f.p, status.p}, nfc, 256, 0, st);
  launch(KBatchGemm{Bf.p, Nf.p, T1.p, d_t1.p, d_gt.p, 0, 1.0, 0.0}, (int64_t)gt.size(), 256, gsm, st);
  launch(KBatchGemm{Nf.p, T1.p, Cf.p, d_t1.p, d_gt.p, 1, 1.0, 0.0}, (int64_t)gt.size(), 256, gsm, st);
  launch(KSymmetrize{Cf.p, d_f.p}, nfc, 256, 0, st);
  int ndmax = 1;
  for (int t = 0; t < nfc; ++t) ndmax = std::max(ndmax, nd[t]);
  launch(KTridiag{Cf.p, DE.p, TAU.p, d_tri.p}, nfc, 256, sizeof(double) * (2 * ndmax + 256), st);
  DBuf<int64_t> d_yo;
  upload_vec(d_yo, yo, st);
  launch(KTridiagEig{Cf.p, DE.p, TAU.p, d_tri.p, b->adapt_theta, MAXSEL, cnt.p, LAM.p, Y.p, d_yo.p}, nfc, 256,
         sizeof(double) * (4 * ndmax + 256 + MAXSEL), st);
  launch(KConstraintRows{Nf.p, Bf.p, Y.p, d_yo.p, d_rows.p, cnt.p, MAXSEL}, nfc, 256, sizeof(double) * ndmax, st);
  const auto stv = status.download(st);
  VB_CHECK(stv[0] == 0, VEM_ESINGULAR, "adaptive: sum of the face Neumann Schur complement inverses not SPD");
  const auto hc = cnt.download(st);
  const auto hy = Y.download(st);
  int added = 0;
  for (int t = 0; t < nfc; ++t) {
    const int g = b->sf_faces[t];
    const Macro& G = b->H.macros[g];
    const int n = (int)G.dofs.size();
    const int m = std::min(hc[t], MAXSEL);
    std::vector<double> c(n), v(n);
    for (int s2 = 0; s2 < m; ++s2) {
      std::fill(c.begin(), c.end(), 0.0);
      for (int k = 0; k < nd[t]; ++k) c[G.r + k] = hy[yo[t] + (int64_t)s2 * nd[t] + k];
      hh_apply(G, c.data(), v.data());
      extra[g].insert(extra[g].end(), v.begin(), v.end());
      ++added;
    }
  }
  return added;
}

}  // namespace vb

using namespace vb;

static int bfail(const Error& e) {
  set_last_error(e.what());
  return e.status;
}

// the whole numeric and symbolic setup of one handle (options already set)
static void setup_core(bddc* b, const int32_t* part) {
    vem_system* s = b->sys;
    cudaStream_t st = b->stream;
    BddcHost& H = b->H;
    auto t0 = std::chrono::steady_clock::now();
    auto mark = [&](const char* name) {
      VB_CUDA(cudaStreamSynchronize(st));
      auto t1 = std::chrono::steady_clock::now();
      b->times.push_back({name, std::chrono::duration<double, std::milli>(t1 - t0).count()});
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        b->times.push_back({std::string("gib_free_after_") + name, (double)fr / (1 << 30)});
      static const bool log = std::getenv("VEMBDDC_SETUP_LOG") != nullptr;
      if (log)
        std::fprintf(stderr, "bddc_setup: %s %.1f ms, %.1f GiB free\n", name, b->times[b->times.size() - 2].second,
                     (double)fr / (1 << 30));
      t0 = std::chrono::steady_clock::now();
    };
    bddc_host_setup(s, part, b->opt, H, s->elem_wmean);
    mark("t_symbolic_ms");
    for (auto& kv : H.times) b->times.push_back(kv);
    const int N = H.N;
    const int np = s->dof.np;
    // ---------------- flatten
    std::vector<int> border, children, rel, dtype, dsrc, bgrp, elpos, elptr, pv, sub_elems, vadj_ptr, vadj, vcon_ptr,
        vcon_id, iface, elloc, elloc_ptr, share, gpos, gif;
    std::vector<int64_t> vdof, press, coarse, mdofs;
    std::vector<double> vcon_coef, wmean, hv, tau, mcon_coef;
    std::vector<int> mcon_ptr, mcon_vdof;
    b->h_subs.assign(N, SubDev{});
    // the per-subdomain tables that need searches, built in parallel:
    // element column -> local index, and the constraint rows by multiplier
    std::vector<std::vector<int>> ell(N), mptr(N), mvd(N);
    std::vector<std::vector<double>> mcoef(N);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < N; ++i) {
      const Subdomain& S = H.subs[i];
      const int nv = (int)S.vdof.size();
      std::vector<int>& el = ell[i];
      for (size_t le = 0; le < S.elems.size(); ++le) {
        const int e = S.elems[le];
        const int nK = (int)(s->h_eoff[e + 1] - s->h_eoff[e]);
        for (int bb = 0; bb < nK; ++bb) {
          const int64_t g = s->h_sysdof[s->h_eoff[e] + bb];
          int l = -1;
          if (g >= 0) l = (int)(std::lower_bound(S.vdof.begin(), S.vdof.end(), g) - S.vdof.begin());
          el.push_back(l);
        }
        for (int a = 0; a < np; ++a) el.push_back(nv + (int)le * np + a);
      }
      int nm = 0;
      for (int id : S.vcon_id) nm = std::max(nm, id + 1);
      std::vector<int> cnt(nm + 1, 0);
      for (int id : S.vcon_id) cnt[id + 1]++;
      for (int m = 0; m < nm; ++m) cnt[m + 1] += cnt[m];
      mptr[i] = cnt;
      mvd[i].assign(cnt[nm], 0);
      mcoef[i].assign(cnt[nm], 0.0);
      for (int v = 0; v < nv; ++v)
        for (int q = S.vcon_ptr[v]; q < S.vcon_ptr[v + 1]; ++q) {
          const int m = S.vcon_id[q];
          mvd[i][cnt[m]] = v;
          mcoef[i][cnt[m]] = S.vcon_coef[q];
          cnt[m]++;
        }
    }
    int64_t loc = 0;
    for (int i = 0; i < N; ++i) {
      const Subdomain& S = H.subs[i];
      SubDev& D = b->h_subs[i];
      D.ne = (int)S.elems.size();
      D.nv = (int)S.vdof.size();
      D.npress = (int)S.press.size();
      D.pstar = S.pstar;
      D.niface = (int)S.iface_vdof.size();
      D.ncl = (int)S.coarse.size();
      D.dir = H.dir_prob[i];
      D.neu = H.neu_prob[i];
      D.volume = S.volume;
      D.wsum = S.volume;   // sum of int_K m_0 over the subdomain = |Omega_i|
      D.elem_off = (int64_t)sub_elems.size();
      sub_elems.insert(sub_elems.end(), S.elems.begin(), S.elems.end());
      D.vdof_off = (int64_t)vdof.size();
      vdof.insert(vdof.end(), S.vdof.begin(), S.vdof.end());
      D.vadj_ptr_off = (int64_t)vadj_ptr.size();
      vadj_ptr.insert(vadj_ptr.end(), S.vadj_ptr.begin(), S.vadj_ptr.end());
      D.vadj_off = (int64_t)vadj.size();
      vadj.insert(vadj.end(), S.vadj.begin(), S.vadj.end());
      D.vcon_ptr_off = (int64_t)vcon_ptr.size();
      vcon_ptr.insert(vcon_ptr.end(), S.vcon_ptr.begin(), S.vcon_ptr.end());
      D.vcon_off = (int64_t)vcon_id.size();
      vcon_id.insert(vcon_id.end(), S.vcon_id.begin(), S.vcon_id.end());
      vcon_coef.insert(vcon_coef.end(), S.vcon_coef.begin(), S.vcon_coef.end());
      // multiplier -> (local vdof, coef): the constraint rows by multiplier
      // (vdofs ascending within a row)
      D.mcon_ptr_off = (int64_t)mcon_ptr.size();
      D.mcon_off = (int64_t)mcon_vdof.size();
      mcon_ptr.insert(mcon_ptr.end(), mptr[i].begin(), mptr[i].end());
      mcon_vdof.insert(mcon_vdof.end(), mvd[i].begin(), mvd[i].end());
      mcon_coef.insert(mcon_coef.end(), mcoef[i].begin(), mcoef[i].end());
      D.press_off = (int64_t)press.size();
      press.insert(press.end(), S.press.begin(), S.press.end());
      wmean.insert(wmean.end(), S.wmean.begin(), S.wmean.end());
      D.iface_off = (int64_t)iface.size();
      iface.insert(iface.end(), S.iface_vdof.begin(), S.iface_vdof.end());
      D.coarse_off = (int64_t)coarse.size();
      coarse.insert(coarse.end(), S.coarse.begin(), S.coarse.end());
      // element column -> local index
      D.ellocptr_off = (int64_t)elloc_ptr.size();
      D.elloc_off = (int64_t)elloc.size();
      int off = 0;
      for (int le = 0; le < D.ne; ++le) {
        elloc_ptr.push_back(off);
        const int e = S.elems[le];
        off += (int)(s->h_eoff[e + 1] - s->h_eoff[e]) + np;
      }
      elloc_ptr.push_back(off);
      elloc.insert(elloc.end(), ell[i].begin(), ell[i].end());
      D.loc_off = loc;
      loc += D.nv + D.npress;
    }
    // problems and nodes: offsets and node records in one pass, then the
    // per-problem tables copied into place in parallel
    b->h_probs.assign(H.probs.size(), ProbDev{});
    b->h_nodes.clear();
    {
      const size_t nq = H.probs.size();
      std::vector<int64_t> o_pos(nq), o_elpos(nq), o_elptr(nq), o_pv(nq), o_bord(nq), o_rel(nq), o_child(nq);
      int64_t n_pos = 0, n_elpos = 0, n_elptr = 0, n_pv = 0, n_bord = 0, n_rel = 0, n_child = 0;
      std::vector<int> nbase(nq);
      for (size_t q = 0; q < nq; ++q) {
        const Problem& P = H.probs[q];
        ProbDev& D = b->h_probs[q];
        D.sub = P.sub;
        D.kind = P.kind;
        D.n = P.n;
        D.npiv = P.npiv;
        D.mult0 = P.mult0;
        D.nmult = P.nmult;
        D.macro = P.macro;
        VB_CHECK(P.bgrp.size() == P.dtype.size() && P.dsrc.size() == P.dtype.size(), VEM_EINVAL,
                 "setup: position tables of a local problem differ in length");
        o_pos[q] = D.pos_off = n_pos;
        n_pos += (int64_t)P.dtype.size();
        o_elpos[q] = D.elpos_off = n_elpos;
        n_elpos += (int64_t)P.elpos.size();
        o_elptr[q] = D.elptr_off = n_elptr;
        n_elptr += (int64_t)P.elpos_off.size();
        o_pv[q] = D.pv_off = n_pv;
        n_pv += (int64_t)P.pos_of_vdof.size();
        o_bord[q] = n_bord;
        n_bord += (int64_t)P.border.size();
        o_rel[q] = n_rel;
        n_rel += (int64_t)P.rel.size();
        o_child[q] = n_child;
        n_child += (int64_t)P.children.size();
        const int base = nbase[q] = (int)b->h_nodes.size();
        for (const Node& Nd : P.nodes) {
          NodeDev N{};
          N.prob = (int)q;
          N.p0 = Nd.p0;
          N.np = Nd.np;
          N.nb = Nd.nb;
          N.parent = Nd.parent >= 0 ? base + Nd.parent : -1;
          N.height = Nd.height;
          N.first_child = (int)o_child[q] + Nd.first_child;
          N.nchild = Nd.nchild;
          N.flags = Nd.flags;
          N.border_off = o_bord[q] + Nd.border_off;
          N.rel_off = o_rel[q] + Nd.rel_off;
          b->h_nodes.push_back(N);
        }
        D.root = (int)b->h_nodes.size() - 1;
      }
      dtype.resize(n_pos);
      bgrp.resize(n_pos);
      dsrc.resize(n_pos);
      elpos.resize(n_elpos);
      elptr.resize(n_elptr);
      pv.resize(n_pv);
      border.resize(n_bord);
      rel.resize(n_rel);
      children.resize(n_child);
#pragma omp parallel for schedule(dynamic)
      for (int64_t q = 0; q < (int64_t)nq; ++q) {
        const Problem& P = H.probs[q];
        std::copy(P.dtype.begin(), P.dtype.end(), dtype.begin() + o_pos[q]);
        std::copy(P.bgrp.begin(), P.bgrp.end(), bgrp.begin() + o_pos[q]);
        for (size_t i = 0; i < P.dsrc.size(); ++i) dsrc[o_pos[q] + i] = (int)P.dsrc[i];
        std::copy(P.elpos.begin(), P.elpos.end(), elpos.begin() + o_elpos[q]);
        std::copy(P.elpos_off.begin(), P.elpos_off.end(), elptr.begin() + o_elptr[q]);
        std::copy(P.pos_of_vdof.begin(), P.pos_of_vdof.end(), pv.begin() + o_pv[q]);
        std::copy(P.border.begin(), P.border.end(), border.begin() + o_bord[q]);
        std::copy(P.rel.begin(), P.rel.end(), rel.begin() + o_rel[q]);
        for (size_t i = 0; i < P.children.size(); ++i) children[o_child[q] + i] = nbase[q] + P.children[i];
      }
    }
    // macro entities; the (entity, sharing subdomain) position and interface
    // index tables need searches and are built in parallel
    const int nmac = (int)H.macros.size();
    std::vector<std::vector<int>> mgpos(nmac), mgif(nmac);
#pragma omp parallel for schedule(dynamic, 16)
    for (int g = 0; g < nmac; ++g) {
      const Macro& G = H.macros[g];
      for (int si : G.share) {
        const Subdomain& S = H.subs[si];
        const Problem& PN = H.probs[H.neu_prob[si]];
        for (int64_t g2 : G.dofs) {
          const int v = (int)(std::lower_bound(S.vdof.begin(), S.vdof.end(), g2) - S.vdof.begin());
          mgpos[g].push_back(PN.pos_of_vdof[v]);
          mgif[g].push_back((int)(std::lower_bound(S.iface_vdof.begin(), S.iface_vdof.end(), v) -
                                  S.iface_vdof.begin()));
        }
      }
    }
    b->h_macros.assign(H.macros.size(), MacroDev{});
    int64_t dual = 0, deluxe_n = 0;
    for (size_t g = 0; g < H.macros.size(); ++g) {
      const Macro& G = H.macros[g];
      MacroDev& D = b->h_macros[g];
      D.kind = G.kind;
      D.n = (int)G.dofs.size();
      D.r = G.r;
      D.nshare = (int)G.share.size();
      D.ndual = D.n - D.r;
      D.dofs_off = (int64_t)mdofs.size();
      mdofs.insert(mdofs.end(), G.dofs.begin(), G.dofs.end());
      if (G.hv.empty()) {
        D.hv_off = -1;
        D.tau_off = -1;
      } else {
        D.hv_off = (int64_t)hv.size();
        hv.insert(hv.end(), G.hv.begin(), G.hv.end());
        D.tau_off = (int64_t)tau.size();
        tau.insert(tau.end(), G.tau.begin(), G.tau.end());
      }
      D.coarse0 = G.coarse0;
      D.dual_off = dual;
      dual += D.ndual;
      D.share_off = (int64_t)share.size();
      share.insert(share.end(), G.share.begin(), G.share.end());
      D.gpos_off = (int64_t)gpos.size();
      D.gif_off = (int64_t)gif.size();
      gpos.insert(gpos.end(), mgpos[g].begin(), mgpos[g].end());
      gif.insert(gif.end(), mgif[g].begin(), mgif[g].end());
      D.deluxe_off = -1;
      D.deluxe_e_off = -1;
    }
    b->ndual = dual;
    // deluxe problems (one per subdomain) and their (problem, entity) tasks
    std::vector<int> dl_probs;
    std::vector<DeluxeTask> dtasks;
    std::vector<int> dtask_prob;   // task -> index into dl_probs
    for (size_t q = 0; q < H.probs.size(); ++q)
      if (H.probs[q].kind == PK_DELUXE) dl_probs.push_back((int)q);
    std::vector<int> faces, edges;
    std::vector<int64_t> sd_i, sd_j, cw_off;
    std::vector<int64_t> e_sd, e_sd_ptr(1, 0);
    int64_t deluxe_e_n = 0, sdn = 0;
    {
      std::map<std::pair<int, int>, int> tq;   // (macro, subdomain) -> task
      for (size_t t = 0; t < dl_probs.size(); ++t) {
        const Problem& HP = H.probs[dl_probs[t]];
        for (size_t m = 0; m < HP.dl_macros.size(); ++m) {
          const MacroDev& G = b->h_macros[HP.dl_macros[m]];
          DeluxeTask tk{dl_probs[t], b->h_probs[dl_probs[t]].root, HP.dl_macros[m], HP.dl_b0[m], 0, sdn};
          sdn += (int64_t)G.ndual * G.ndual;
          tq[{HP.dl_macros[m], HP.sub}] = (int)dtasks.size();
          dtasks.push_back(tk);
          dtask_prob.push_back((int)t);
        }
      }
      for (size_t g = 0; g < H.macros.size(); ++g) {
        MacroDev& G = b->h_macros[g];
        if (G.kind != 2 || G.ndual == 0) continue;
        auto ia = tq.find({(int)g, H.macros[g].share[0]});
        auto ib = tq.find({(int)g, H.macros[g].share[1]});
        if (ia == tq.end() || ib == tq.end()) continue;
        faces.push_back((int)g);
        sd_i.push_back(dtasks[ia->second].sd_off);
        sd_j.push_back(dtasks[ib->second].sd_off);
        G.deluxe_off = deluxe_n;
        deluxe_n += (int64_t)G.ndual * G.ndual;
      }
      int64_t c = 0;
      for (int g : faces) {
        cw_off.push_back(c);
        c += (int64_t)b->h_macros[g].ndual * b->h_macros[g].ndual;
      }
      // deluxe edges: the dual blocks of all sharing subdomains, in the
      // order of the entity's sharing list
      if (b->opt.scaling == BDDC_SCALING_DELUXE_EDGES) {
        for (size_t g = 0; g < H.macros.size(); ++g) {
          MacroDev& G = b->h_macros[g];
          if (G.kind != 1 || G.ndual == 0) continue;
          std::vector<int64_t> offs;
          for (int sd : H.macros[g].share) {
            auto it = tq.find({(int)g, sd});
            if (it == tq.end()) break;
            offs.push_back(dtasks[it->second].sd_off);
          }
          if (offs.size() != H.macros[g].share.size()) continue;
          edges.push_back((int)g);
          e_sd.insert(e_sd.end(), offs.begin(), offs.end());
          e_sd_ptr.push_back((int64_t)e_sd.size());
          G.deluxe_e_off = deluxe_e_n;
          deluxe_e_n += (int64_t)G.nshare * G.ndual * G.ndual;
        }
      }
    }
    mark("t_flatten_ms");
    // ---------------- upload structure
    upload_vec(b->d_border, border, st);
    upload_vec(b->d_children, children, st);
    upload_vec(b->d_rel, rel, st);
    upload_vec(b->d_dtype, dtype, st);
    upload_vec(b->d_bgrp, bgrp, st);
    upload_vec(b->d_dsrc, dsrc, st);
    upload_vec(b->d_elpos, elpos, st);
    upload_vec(b->d_elptr, elptr, st);
    upload_vec(b->d_pv, pv, st);
    upload_vec(b->d_sub_elems, sub_elems, st);
    upload_vec(b->d_vadj_ptr, vadj_ptr, st);
    upload_vec(b->d_vadj, vadj, st);
    upload_vec(b->d_vcon_ptr, vcon_ptr, st);
    upload_vec(b->d_vcon_id, vcon_id, st);
    upload_vec(b->d_vcon_coef, vcon_coef, st);
    upload_vec(b->d_iface, iface, st);
    upload_vec(b->d_elloc, elloc, st);
    upload_vec(b->d_elloc_ptr, elloc_ptr, st);
    upload_vec(b->d_share, share, st);
    upload_vec(b->d_gpos, gpos, st);
    upload_vec(b->d_gif, gif, st);
    upload_vec(b->d_vdof, vdof, st);
    upload_vec(b->d_press, press, st);
    upload_vec(b->d_coarse, coarse, st);
    upload_vec(b->d_mdofs, mdofs, st);
    upload_vec(b->d_wmean, wmean, st);
    upload_vec(b->d_hv, hv, st);
    upload_vec(b->d_tau, tau, st);
    upload_vec(b->d_mcon_ptr, mcon_ptr, st);
    upload_vec(b->d_mcon_vdof, mcon_vdof, st);
    upload_vec(b->d_mcon_coef, mcon_coef, st);
    b->ncv = H.ncoarse_vel;
    b->nc = H.ncoarse;
    // batches
    std::vector<int> dprobs(H.dir_prob.begin(), H.dir_prob.end()), nprobs(H.neu_prob.begin(), H.neu_prob.end());
    build_batch(b, b->bd, dprobs, true);
    build_batch(b, b->bn, nprobs, true);
    upload_vec(b->d_fvoff, b->h_fvoff, st);
    b->times.push_back({"gflop_factor_dirichlet", batch_gflop(b, dprobs)});
    b->times.push_back({"gflop_factor_neumann", batch_gflop(b, nprobs)});
    b->times.push_back({"gflop_factor_deluxe", batch_gflop(b, dl_probs)});
    upload_vec(b->d_nodes, b->h_nodes, st);
    upload_vec(b->d_probs, b->h_probs, st);
    upload_vec(b->d_subs, b->h_subs, st);
    upload_vec(b->d_macros, b->h_macros, st);
    upload_levels(b, b->bd);
    upload_levels(b, b->bn);
    if (b->prec == 1) {
      // element matrices as FP32 (high, low) pairs for the refinement residual
      const int64_t na = (int64_t)s->d_A.n;
      b->d_A2.alloc(na);
      launch(KSplitPairs{s->d_A.p, b->d_A2.p, na}, (na + 255) / 256, 256, 0, st);
    }
    BddcView V = make_view(b);
    mark("t_upload_ms");
    // ---------------- numeric factorizations (S4)
    DBuf<int> status(1);
    status.zero(st);
    // the update matrices are consumed by the parents during the
    // factorization and not needed afterwards: released batch by batch
    // Dirichlet factors: taken from the deluxe factorization when every
    // subdomain has a deluxe problem with the same pivots, tree and leading
    // border (checked here), else factored
    std::vector<PanelCopyTask> pcopy;       // per deluxe problem, in dl_probs order
    std::vector<int64_t> pcopy_ptr(1, 0);
    {
      bool from_dl = !dl_probs.empty() && (int)dl_probs.size() == N;
      std::vector<int> dl_of_sub(N, -1);
      if (from_dl)
        for (int q : dl_probs) {
          const int i = H.probs[q].sub;
          if (dl_of_sub[i] >= 0) from_dl = false;
          else dl_of_sub[i] = q;
        }
      for (int i = 0; i < N && from_dl; ++i) {
        const Problem& PD = H.probs[H.dir_prob[i]];
        const Problem& PX = H.probs[dl_of_sub[i]];
        if (PD.npiv != PX.npiv || PD.nodes.size() != PX.nodes.size()) { from_dl = false; break; }
        for (size_t k = 0; k < PD.nodes.size() && from_dl; ++k) {
          const Node &nd = PD.nodes[k], &nx = PX.nodes[k];
          if (nd.p0 != nx.p0 || nd.np != nx.np || nd.nb > nx.nb || nd.nchild != nx.nchild) { from_dl = false; break; }
          for (int j = 0; j < nd.nb; ++j)
            if (PD.border[nd.border_off + j] != PX.border[nx.border_off + j]) { from_dl = false; break; }
        }
      }
      if (from_dl) {
        for (int q : dl_probs) {
          const int i = H.probs[q].sub;
          const int nn = (int)H.probs[q].nodes.size();
          const int rd = b->h_probs[H.dir_prob[i]].root - nn + 1, rx = b->h_probs[q].root - nn + 1;
          for (int k = 0; k < nn; ++k)
            for (int c0 = 0; c0 < b->h_nodes[rd + k].np; c0 += 32) pcopy.push_back({rd + k, rx + k, c0});
          pcopy_ptr.push_back((int64_t)pcopy.size());
        }
        if (b->prec == 0) b->bd.F.alloc(std::max<int64_t>(b->bd.nF, 1));
        else b->bd.F32.alloc(std::max<int64_t>(b->bd.nF, 1));
      } else {
        pcopy_ptr.clear();
        factor_batch(b, b->bd, V, status);
        VB_CUDA(cudaStreamSynchronize(st));
        b->bd.U.release();
        b->bd.U32.release();
      }
    }
    mark("t_factor_dirichlet_ms");
    factor_batch(b, b->bn, V, status);
    VB_CUDA(cudaStreamSynchronize(st));
    b->bn.U.release();
    b->bn.U32.release();
    mark("t_factor_neumann_ms");
    {
      auto stv = status.download(st);
      VB_CHECK(stv[0] != 2, VEM_EINVAL, "local factorization: matrix entry outside the symbolic front");
      VB_CHECK(stv[0] == 0, VEM_ESINGULAR, "local factorization: zero or wrong-signed pivot");
    }
    // ---------------- deluxe blocks (S6): one problem per subdomain (the
    // Dirichlet pivots with all its deluxe entities' DOFs at the root),
    // factored in chunks of bounded memory; the root update matrix holds
    // every entity's block S_FF, each rotated to the dual coordinates and
    // kept, the partial factors are released
    b->d_deluxe.alloc(std::max<int64_t>(deluxe_n, 1));
    b->d_deluxe_e.alloc(std::max<int64_t>(deluxe_e_n, 1));
    if (!faces.empty() || !edges.empty()) {
      DBuf<double> SD(std::max<int64_t>(sdn, 1));
      const double budget = 96.0 * (1 << 30);
      const double vbytes = b->prec == 0 ? 8.0 : 4.0;
      size_t t0c = 0, k0c = 0;   // first problem and first task of the chunk
      while (t0c < dl_probs.size()) {
        double bytes = 0;
        size_t t1c = t0c;
        while (t1c < dl_probs.size()) {
          const Problem& HP = H.probs[dl_probs[t1c]];
          double pb = 0;
          for (const Node& Nd : HP.nodes) pb += vbytes * ((double)(Nd.np + Nd.nb) * Nd.np + (double)Nd.nb * Nd.nb);
          for (int g : HP.dl_macros) pb += 8.0 * b->h_macros[g].n * b->h_macros[g].n;
          if (t1c > t0c && bytes + pb > budget) break;
          bytes += pb;
          ++t1c;
        }
        std::vector<int> cp(dl_probs.begin() + t0c, dl_probs.begin() + t1c);
        size_t k1c = k0c;
        int64_t w = 0;
        std::vector<DeluxeTask> ct;
        while (k1c < dtasks.size() && dtask_prob[k1c] < (int)t1c) {
          DeluxeTask tk = dtasks[k1c++];
          tk.work_off = w;
          w += (int64_t)b->h_macros[tk.macro].n * b->h_macros[tk.macro].n;
          ct.push_back(tk);
        }
        Batch Bc;
        build_batch(b, Bc, cp, false);
        upload_vec(b->d_nodes, b->h_nodes, st);
        upload_levels(b, Bc);
        V = make_view(b);
        factor_batch(b, Bc, V, status);
        if (!pcopy_ptr.empty() && pcopy_ptr[t1c] > pcopy_ptr[t0c]) {
          DBuf<PanelCopyTask> dpc;
          std::vector<PanelCopyTask> pc(pcopy.begin() + pcopy_ptr[t0c], pcopy.begin() + pcopy_ptr[t1c]);
          upload_vec(dpc, pc, st);
          if (b->prec == 0)
            launch(KPanelCopy<double>{V, dpc.p, Bc.F.p, b->bd.F.p}, (int64_t)pc.size(), 256, 0, st);
          else
            launch(KPanelCopy<float>{V, dpc.p, Bc.F32.p, b->bd.F32.p}, (int64_t)pc.size(), 256, 0, st);
          VB_CUDA(cudaStreamSynchronize(st));
        }
        DBuf<DeluxeTask> dct;
        upload_vec(dct, ct, st);
        DBuf<double> work(std::max<int64_t>(w, 1));
        if (b->prec == 0)
          launch(KDeluxeExtract<double>{V, dct.p, Bc.U.p, work.p, SD.p}, (int)ct.size(), 256, 0, st);
        else
          launch(KDeluxeExtract<float>{V, dct.p, Bc.U32.p, work.p, SD.p}, (int)ct.size(), 256, 0, st);
        VB_CUDA(cudaStreamSynchronize(st));
        t0c = t1c;
        k0c = k1c;
      }
      {
        auto stv = status.download(st);
        VB_CHECK(stv[0] != 2, VEM_EINVAL, "deluxe factorization: entry outside the symbolic front");
        VB_CHECK(stv[0] == 0, VEM_ESINGULAR, "deluxe factorization: zero or wrong-signed pivot");
      }
      mark("t_factor_deluxe_ms");
      if (!faces.empty()) {
        DBuf<int> df;
        DBuf<int64_t> dsi, dsj, dpo, duo;
        std::vector<int64_t> po, uo;
        std::vector<GemmTile> tiles;
        int64_t pn = 0, un = 0;
        for (size_t t = 0; t < faces.size(); ++t) {
          const int nd = b->h_macros[faces[t]].ndual;
          po.push_back(pn);
          pn += (int64_t)2 * nd * nd;
          uo.push_back(un);
          un += (int64_t)nd * nd;
          const int nt = (nd + 63) / 64;
          for (int ti = 0; ti < nt; ++ti)
            for (int tj = 0; tj < nt; ++tj) tiles.push_back({(int)t, ti, tj});
        }
        upload_vec(df, faces, st);
        upload_vec(dsi, sd_i, st);
        upload_vec(dsj, sd_j, st);
        upload_vec(dpo, po, st);
        upload_vec(duo, uo, st);
        DBuf<GemmTile> dtiles;
        upload_vec(dtiles, tiles, st);
        DBuf<double> PAN(std::max<int64_t>(pn, 1)), UPD(std::max<int64_t>(un, 1));
        V = make_view(b);
        // one CTA per face, four groups of 256 threads on separate trailing tiles
        int ndmax = 0;
        for (int g : faces) ndmax = std::max(ndmax, b->h_macros[g].ndual);
        launch_mt<1024>(KDeluxeFront{V, df.p, dsi.p, dsj.p, SD.p, PAN.p, UPD.p, dpo.p, duo.p, status.p}, (int)faces.size(), 1024,
               sizeof(double) * (std::max(4 * 2 * 64 * 32 + 128, ndmax) + 8), st);
        launch(KDeluxeGemm{V, dtiles.p, df.p, PAN.p, dpo.p, b->d_deluxe.p}, (int64_t)tiles.size(), 256,
               sizeof(double) * (2 * 32 * 64 + 8), st);
        mark("t_deluxe_combine_ms");
        auto stv = status.download(st);
        VB_CHECK(stv[0] == 0, VEM_ESINGULAR, "deluxe: face Schur complement sum not positive definite");
      }
      if (!edges.empty()) {
        // deluxe edges: W = sum_s S_s, W = G G^T, D_s = W^{-1} S_s
        std::vector<DenseItem> items;
        std::vector<int64_t> wo;
        std::vector<int> te, ts;
        int64_t wn = 0;
        for (size_t t = 0; t < edges.size(); ++t) {
          const MacroDev& G = b->h_macros[edges[t]];
          wo.push_back(wn);
          items.push_back({G.ndual, wn, 0, 0});
          wn += (int64_t)G.ndual * G.ndual;
          for (int q = 0; q < G.nshare; ++q) {
            te.push_back((int)t);
            ts.push_back(q);
          }
        }
        DBuf<int> de, dte, dts, est(1);
        DBuf<int64_t> desp, deso, dewo;
        DBuf<DenseItem> dit;
        upload_vec(de, edges, st);
        upload_vec(dte, te, st);
        upload_vec(dts, ts, st);
        upload_vec(desp, e_sd_ptr, st);
        upload_vec(deso, e_sd, st);
        upload_vec(dewo, wo, st);
        upload_vec(dit, items, st);
        DBuf<double> WE(std::max<int64_t>(wn, 1));
        est.zero(st);
        V = make_view(b);
        launch(KDeluxeEdgeSum{V, de.p, desp.p, deso.p, SD.p, WE.p, dewo.p}, (int)edges.size(), 256, 0, st);
        launch(KCholesky{WE.p, dit.p, est.p}, (int)edges.size(), 256, 0, st);
        auto ev = est.download(st);
        VB_CHECK(ev[0] == 0, VEM_ESINGULAR, "deluxe: edge Schur complement sum not positive definite");
        launch(KDeluxeEdgeSolve{V, de.p, dte.p, dts.p, desp.p, deso.p, SD.p, WE.p, dewo.p, b->d_deluxe_e.p},
               (int64_t)te.size(), 256, 0, st);
        VB_CUDA(cudaStreamSynchronize(st));
        mark("t_deluxe_edges_ms");
      }
      if (b->keep_sf) {
        b->d_sf = std::move(SD);
        b->sf_faces = faces;
        b->sf_i = sd_i;
        b->sf_j = sd_j;
      }
    }
    upload_vec(b->d_macros, b->h_macros, st);
    V = make_view(b);
    // ---------------- coarse basis and coarse matrix (S5)
    int NC = 1;
    for (auto& S : b->h_subs) NC = std::max(NC, S.ncl);
    {
      // W on the device: the primal columns H e_q of every (entity, sharing
      // subdomain) pair, then the p_0 columns
      std::vector<CoarseWTask> wt;
      for (int i = 0; i < N; ++i) {
        const Subdomain& S = H.subs[i];
        int c = 0;
        for (int gi : S.macros) {
          const Macro& G = H.macros[gi];
          const int si = (int)(std::find(G.share.begin(), G.share.end(), i) - G.share.begin());
          VB_CHECK(si < (int)G.share.size(), VEM_EINVAL, "coarse basis: entity not shared by its subdomain");
          if (G.r > 0) wt.push_back({gi, si, c});
          c += G.r;
        }
        VB_CHECK(c + 1 == b->h_subs[i].ncl, VEM_EINVAL, "coarse column count mismatch");
      }
      DBuf<double> dW((size_t)loc * NC), KW((size_t)loc * NC), PHI((size_t)loc * NC);
      DBuf<int2> wcols(std::max<int64_t>(loc, 1));
      dW.zero(st);
      wcols.zero(st);
      {
        DBuf<CoarseWTask> dwt;
        upload_vec(dwt, wt, st);
        if (!wt.empty())
          launch(KCoarseW{V, dwt.p, dW.p, wcols.p, NC}, (int64_t)wt.size(), 256,
                 sizeof(double) * (max_macro_n(b) + 256 + 8), st);
        launch(KCoarseWP0{V, dW.p, wcols.p, NC}, N, 256, 0, st);
        VB_CUDA(cudaStreamSynchronize(st));
      }
      std::vector<int64_t> rp(N + 1, 0);
      for (int i = 0; i < N; ++i) rp[i + 1] = rp[i] + b->h_subs[i].nv + b->h_subs[i].npress;
      DBuf<int64_t> drp;
      upload_vec(drp, rp, st);
      KW.zero(st);
      launch(KElemMatvecW{V, drp.p, N, dW.p, wcols.p, KW.p, NC}, loc, 32, sizeof(double) * NC, st);
      mark("t_coarse_rhs_ms");
      // constrained Neumann solves for the coarse basis, CH columns at a time
      // (the right-hand-side, front-vector and refinement stores scale with CH)
      const int CH = std::min(NC, 64);
      b->XN.alloc(std::max<int64_t>(b->bn.vec_n * CH, 1));
      b->UVN.alloc(std::max<int64_t>(b->bn.uvec_n * CH, 1));
      for (int c0 = 0; c0 < NC; c0 += CH) {
        const int ch = std::min(CH, NC - c0);
        launch(KNeuRhsPhi{V, KW.p, b->XN.p, NC, c0, ch}, (int64_t)N * ch, 256, sizeof(double) * 256, st);
        solve_batch(b, b->bn, V, b->XN.p, b->UVN.p, ch);
        launch(KPhiAssemble{V, dW.p, b->XN.p, PHI.p, NC, c0, ch}, (int64_t)N * ch, 256, sizeof(double) * 256, st);
      }
      mark("t_coarse_solves_ms");
      // K Phi with Phi and the product row-major (coalesced over columns):
      // the Phi copy takes the buffer of W, the product that of K W
      if (V.A2) {
        launch(KToRowMajor<true>{drp.p, N, loc, PHI.p, dW.p, NC}, (loc + 31) / 32, 256, sizeof(double) * 32 * 33, st);
        launch(KElemMatvecRM<true>{V, drp.p, N, dW.p, KW.p, NC}, loc, 32, 0, st);
      } else {
        launch(KToRowMajor<false>{drp.p, N, loc, PHI.p, dW.p, NC}, (loc + 31) / 32, 256, sizeof(double) * 32 * 33, st);
        launch(KElemMatvecRM<false>{V, drp.p, N, dW.p, KW.p, NC}, loc, 32, 0, st);
      }
      DBuf<double> SG((size_t)N * NC * NC);
      {
        std::vector<GramTile> gt;
        for (int i = 0; i < N; ++i)
          for (int a0 = 0; a0 < b->h_subs[i].ncl; a0 += 32)
            for (int b0 = 0; b0 < b->h_subs[i].ncl; b0 += 32) gt.push_back({i, a0, b0});
        DBuf<GramTile> dgt;
        upload_vec(dgt, gt, st);
        launch(KGramTiled{V, dgt.p, PHI.p, KW.p, SG.p, NC}, (int64_t)gt.size(), 256,
               sizeof(double) * 2 * KGramTiled::TR * KGramTiled::TP, st);
        VB_CUDA(cudaStreamSynchronize(st));
      }
      mark("t_coarse_gram_ms");
      int64_t nphi = 0;
      for (auto& D : b->h_subs) {
        D.phi_off = nphi;
        nphi += (int64_t)D.niface * D.ncl;
      }
      upload_vec(b->d_subs, b->h_subs, st);
      V = make_view(b);
      b->d_phi.alloc(std::max<int64_t>(nphi, 1));
      launch(KPhiGamma{V, PHI.p, b->d_phi.p, NC}, N, 256, 0, st);
      const int64_t nb = b->nc + 1;
      DBuf<double> KB(nb * nb);
      b->d_Kinv.alloc(nb * nb);
      launch(KCoarseAssemble{V, SG.p, KB.p, N, NC}, 1, 256, 0, st);
      status.zero(st);
      {
        std::vector<double> eye(nb * nb, 0.0);
        for (int64_t q = 0; q < nb; ++q) eye[q * nb + q] = 1.0;
        b->d_Kinv.upload(eye, st);
        const int rows = 8;
        for (int64_t c = 0; c < nb; ++c) {
          launch(KGJPivot{KB.p, b->d_Kinv.p, nb, c, status.p}, 1, 256, sizeof(double) * 512, st);
          launch(KGJElim{KB.p, b->d_Kinv.p, nb, c, rows}, (nb + rows - 1) / rows, 256, 0, st);
        }
      }
      mark("t_coarse_inverse_ms");
      auto stv = status.download(st);
      VB_CHECK(stv[0] == 0, VEM_ESINGULAR, "coarse matrix singular");
    }
    // coarse gather lists
    {
      std::vector<std::vector<std::pair<int, int>>> lists(b->nc);
      for (int i = 0; i < N; ++i)
        for (int c = 0; c < b->h_subs[i].ncl; ++c) lists[H.subs[i].coarse[c]].push_back({i, c});
      std::vector<int> ptr(b->nc + 1, 0), sub, lc;
      for (int64_t c = 0; c < b->nc; ++c) {
        for (auto& pr : lists[c]) { sub.push_back(pr.first); lc.push_back(pr.second); }
        ptr[c + 1] = (int)sub.size();
      }
      upload_vec(b->d_cg_ptr, ptr, st);
      upload_vec(b->d_cg_sub, sub, st);
      upload_vec(b->d_cg_loc, lc, st);
    }
    // ---------------- apply workspaces
    b->XN.alloc(std::max<int64_t>(b->bn.vec_n, 1));
    b->UVN.alloc(std::max<int64_t>(b->bn.uvec_n, 1));
    b->XD.alloc(std::max<int64_t>(b->bd.vec_n, 1));
    b->UVD.alloc(std::max<int64_t>(b->bd.uvec_n, 1));
    b->rC.alloc(b->nc + 1);
    b->uC.alloc(b->nc + 1);
    b->cloc.alloc((size_t)N * NC);
    int64_t nif = 0;
    for (auto& D : b->h_subs) nif += D.niface;
    b->wloc.alloc(std::max<int64_t>(nif, 1));
    b->dwork.alloc(std::max<int64_t>(b->ndual, 1));
    b->dtw.alloc(std::max<int64_t>(b->ndual, 1));
    b->wd1.alloc(std::max<int64_t>(b->ndual, 1));
    b->avgd.alloc(std::max<int64_t>(b->ndual, 1));
    b->NC = NC;
    b->h_dtT.clear();
    b->h_dtN.clear();
    for (size_t g = 0; g < b->h_macros.size(); ++g) {
      const MacroDev& G = b->h_macros[g];
      if (G.deluxe_off < 0) continue;
      b->max_nd = std::max(b->max_nd, G.ndual);
      for (int k0 = 0; k0 < G.ndual; k0 += 64) b->h_dtT.push_back({(int)g, k0});
      for (int k0 = 0; k0 < G.ndual; k0 += 256) b->h_dtN.push_back({(int)g, k0});
    }
    b->h_ift.clear();
    for (int i = 0; i < N; ++i)
      for (int l0 = 0; l0 < b->h_subs[i].niface; l0 += 256) b->h_ift.push_back({i, l0});
    upload_vec(b->d_dtT, b->h_dtT, st);
    upload_vec(b->d_dtN, b->h_dtN, st);
    upload_vec(b->d_ift, b->h_ift, st);
    b->y.alloc(s->n);
    b->part.alloc(b->h_macros.size() + N + 1024 + 8);
    b->r.alloc(s->n);
    b->z.alloc(s->n);
    b->p.alloc(s->n);
    b->Ap.alloc(s->n);
    b->scal.alloc(4);
    VB_CUDA(cudaStreamSynchronize(st));
}

// options of bddc_setup into a fresh handle
static void configure(bddc* b, vem_system* s, uint32_t constraints, int scaling, const bddc_options* opts) {
  b->sys = s;
  b->stream = s->stream;
  b->opt.constraints = constraints;
  VB_CHECK(scaling >= BDDC_SCALING_MULTIPLICITY && scaling <= BDDC_SCALING_DELUXE_EDGES, VEM_EINVAL,
           "bddc_setup: scaling must be 0 (multiplicity), 1 (deluxe faces) or 2 (deluxe faces and edges)");
  b->opt.scaling = scaling;
  if (!opts) return;
  if (opts->nd_leaf > 0) b->opt.leaf = opts->nd_leaf;
  VB_CHECK(opts->use_graph >= -1 && opts->use_graph <= 1, VEM_EINVAL, "bddc_options.use_graph must be -1, 0 or 1");
  b->use_graph = opts->use_graph >= 0;
  VB_CHECK(opts->precision >= 0 && opts->precision <= 2, VEM_EINVAL, "bddc_options.precision must be 0, 1 or 2");
  b->prec = opts->precision;
  VB_CHECK(opts->refine >= 0 && opts->refine <= 4, VEM_EINVAL, "bddc_options.refine must be 0..4");
  if (opts->refine > 0) b->refine = opts->refine;
  VB_CHECK(opts->tc_update >= -1 && opts->tc_update <= 1, VEM_EINVAL, "bddc_options.tc_update must be -1, 0 or 1");
  b->use_tc = opts->tc_update > 0;
  VB_CHECK(opts->adaptive_threshold >= 0.0, VEM_EINVAL, "bddc_options.adaptive_threshold must be >= 0");
  b->adapt_theta = opts->adaptive_threshold;
}

extern "C" int bddc_setup(vem_system* s, const int32_t* part, uint32_t constraints, int scaling,
                          const bddc_options* opts, bddc** out) {
  if (!s || !part || !out) { set_last_error("bddc_setup: null argument"); return VEM_EINVAL; }
  *out = nullptr;
  bddc* b = new bddc();
  try {
    configure(b, s, constraints, scaling, opts);
    const bool adaptive = b->adapt_theta > 0.0 && scaling >= BDDC_SCALING_DELUXE && !(constraints & BDDC_ALL);
    b->keep_sf = adaptive;
    setup_core(b, part);
    if (adaptive) {
      // Sec. 6: eigenvector-based primal rows per macro face, then the whole
      // setup again with the enlarged primal space
      auto t0 = std::chrono::steady_clock::now();
      std::vector<std::vector<double>> extra;
      const int added = adaptive_rows(b, extra);
      const double t_eig = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      std::vector<std::pair<std::string, double>> t1 = b->times;
      if (added > 0) {
        delete b;
        b = nullptr;
        b = new bddc();
        configure(b, s, constraints, scaling, opts);
        b->opt.extra = std::move(extra);
        setup_core(b, part);
        for (auto& pr : t1) b->times.push_back({"first_" + pr.first, pr.second});
      }
      b->times.push_back({"t_adaptive_eig_ms", t_eig});
      b->n_adaptive = added;
    }
    *out = b;
    return VEM_OK;
  } catch (const Error& e) {
    delete b;
    return bfail(e);
  } catch (const std::exception& e) {
    delete b;
    set_last_error(e.what());
    return VEM_ENOMEM;
  }
}

extern "C" int bddc_apply(bddc* b, const double* r, double* z) {
  if (!b || !r || !z) { set_last_error("bddc_apply: null argument"); return VEM_EINVAL; }
  try {
    if (b->use_graph) apply_graph(b, r, z);
    else apply_bddc(b, r, z);
    return VEM_OK;
  } catch (const Error& e) {
    return bfail(e);
  }
}

extern "C" int pcg_solve(bddc* b, const double* f, double* u, double rtol, int maxit, int* iters, double* kappa,
                         double* lam_min, double* lam_max) {
  if (!b || !f || !u) { set_last_error("pcg_solve: null argument"); return VEM_EINVAL; }
  if (maxit < 0) { set_last_error("pcg_solve: maxit < 0"); return VEM_EINVAL; }
  try {
    vem_system* s = b->sys;
    const int64_t n = s->n;
    cudaStream_t st = b->stream;
    const BddcView V = make_view(b);
    const int N = b->H.N;
    const int nblk = (int)((n + 255) / 256);
    // the graph form iterates on a private copy of u (its addresses are
    // captured once per handle)
    if (b->use_graph && (int64_t)b->xg.n != n) { invalidate_graphs(b); b->xg.alloc(n); }
    double* x = b->use_graph ? b->xg.p : u;
    // x0: interior Dirichlet solves, zero interface data
    VB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    launch(KDirRhs{V, f, 1.0, b->XD.p}, N, 256, sizeof(double) * 256, st);
    solve_batch(b, b->bd, V, b->XD.p, b->UVD.p, 1);
    launch(KDirOut{V, b->XD.p, nullptr, x}, N, 256, sizeof(double) * 256, st);
    spmv(s, x, b->Ap.p, st);
    launch(KSub{f, b->Ap.p, b->r.p, n}, nblk, 256, 0, st);
    const double n0 = iface_norm(b, b->r.p);
    const double nf = std::sqrt(dot(b, f, f, n));
    std::vector<double> al, be;
    int it = 0;
    int status = VEM_OK;
    if (!std::isfinite(n0) || !std::isfinite(nf)) {
      // a non-finite right-hand side or initial residual: no iteration
      status = VEM_EBREAKDOWN;
    } else if (n0 > 1e-14 * nf && maxit == 0) {
      status = VEM_ENOTCONV;
    } else if (n0 > 1e-14 * nf && b->use_graph) {
      // the whole loop as one graph launch: a conditional while node runs
      // one iteration per pass until the device-side stop rule clears it
      if (b->pcg_cap < maxit || !b->pcg_exec) {
        if (b->pcg_cap < maxit || !b->pcg_s.p) {
          invalidate_graphs(b);
          b->pcg_cap = std::max(maxit, 64);
          b->pcg_al.alloc(b->pcg_cap);
          b->pcg_be.alloc(b->pcg_cap);
          b->pcg_s.alloc(PS_COUNT);
        }
        pcg_capture(b);
      }
      double hs[PS_COUNT] = {};
      hs[PS_TOL] = rtol * n0;
      hs[PS_MAXIT] = maxit;
      VB_CUDA(cudaMemcpyAsync(b->pcg_s.p, hs, sizeof hs, cudaMemcpyHostToDevice, st));
      VB_CUDA(cudaMemsetAsync(b->p.p, 0, sizeof(double) * n, st));
      VB_CUDA(cudaGraphLaunch(b->pcg_exec, st));
      VB_CUDA(cudaMemcpyAsync(hs, b->pcg_s.p, sizeof hs, cudaMemcpyDeviceToHost, st));
      VB_CUDA(cudaStreamSynchronize(st));
      it = (int)hs[PS_IT];
      const int ps = (int)hs[PS_STATUS];
      status = ps == 1 ? VEM_OK : (ps == 2 ? VEM_EBREAKDOWN : VEM_ENOTCONV);
      g_launches.fetch_add(b->pcg_body_launches * (it + (ps == 2 ? 1 : 0)));
      al.resize(it);
      be.resize(it > 0 ? it - 1 : 0);
      if (it > 0) VB_CUDA(cudaMemcpyAsync(al.data(), b->pcg_al.p, sizeof(double) * it, cudaMemcpyDeviceToHost, st));
      if (it > 1) VB_CUDA(cudaMemcpyAsync(be.data(), b->pcg_be.p, sizeof(double) * (it - 1), cudaMemcpyDeviceToHost, st));
      VB_CUDA(cudaStreamSynchronize(st));
    } else if (n0 > 1e-14 * nf) {
      // host-driven loop: the scalars come back to the host every iteration
      apply_bddc(b, b->r.p, b->z.p);
      VB_CUDA(cudaMemcpyAsync(b->p.p, b->z.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      double rz = dot(b, b->r.p, b->z.p, n);
      status = VEM_ENOTCONV;
      while (it < maxit) {
        spmv(s, b->p.p, b->Ap.p, st);
        const double pAp = dot(b, b->p.p, b->Ap.p, n);
        if (!(pAp > 0.0) || !std::isfinite(pAp) || !std::isfinite(rz)) { status = VEM_EBREAKDOWN; break; }
        const double alpha = rz / pAp;
        launch(KAxpby{b->p.p, x, alpha, 1.0, n}, nblk, 256, 0, st);
        launch(KAxpby{b->Ap.p, b->r.p, -alpha, 1.0, n}, nblk, 256, 0, st);
        ++it;
        al.push_back(alpha);
        const double nr = iface_norm(b, b->r.p);
        if (nr <= rtol * n0) { status = VEM_OK; break; }
        apply_bddc(b, b->r.p, b->z.p);
        const double rzn = dot(b, b->r.p, b->z.p, n);
        const double beta = rzn / rz;
        be.push_back(beta);
        rz = rzn;
        launch(KAxpby{b->z.p, b->p.p, 1.0, beta, n}, nblk, 256, 0, st);
      }
    }
    if (x != u) VB_CUDA(cudaMemcpyAsync(u, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double lmin = 1.0, lmax = 1.0;
    lanczos(al, be, lmin, lmax);
    if (iters) *iters = it;
    if (lam_min) *lam_min = lmin;
    if (lam_max) *lam_max = lmax;
    if (kappa) *kappa = lmax / lmin;
    VB_CUDA(cudaStreamSynchronize(st));
    if (status != VEM_OK)
      set_last_error(status == VEM_ENOTCONV ? "CG did not reach rtol"
                                            : "CG breakdown (p^T K p <= 0, or a non-finite residual)");
    return status;
  } catch (const Error& e) {
    return bfail(e);
  }
}

extern "C" int bddc_set_stream(bddc* b, void* st) {
  if (!b) { set_last_error("null bddc"); return VEM_EINVAL; }
  b->stream = (cudaStream_t)st;
  return VEM_OK;
}

extern "C" int bddc_info(bddc* b, const char* key, double* value) {
  if (!b || !key || !value) { set_last_error("bddc_info: null argument"); return VEM_EINVAL; }
  std::string k(key);
  if (k == "n_subdomains") *value = b->H.N;
  else if (k == "n_coarse") *value = (double)b->nc;
  else if (k == "n_macro") *value = (double)b->h_macros.size();
  else if (k == "factor_bytes_dirichlet") *value = (b->prec ? 4.0 : 8.0) * b->bd.nF;
  else if (k == "factor_bytes_neumann") *value = (b->prec ? 4.0 : 8.0) * b->bn.nF;
  else if (k == "n_deluxe_faces") {
    int c = 0;
    for (auto& G : b->h_macros) c += G.deluxe_off >= 0;
    *value = c;
  } else if (k == "deluxe_bytes") {
    double t = 0;
    for (auto& G : b->h_macros)
      if (G.deluxe_off >= 0) t += 8.0 * G.ndual * G.ndual;
    *value = t;
  } else if (k == "n_deluxe_edges") {
    int c = 0;
    for (auto& G : b->h_macros) c += G.deluxe_e_off >= 0;
    *value = c;
  } else if (k == "deluxe_edge_bytes") {
    double t = 0;
    for (auto& G : b->h_macros)
      if (G.deluxe_e_off >= 0) t += 8.0 * G.nshare * G.ndual * G.ndual;
    *value = t;
  } else if (k == "phi_bytes") *value = 8.0 * b->d_phi.n;
  else if (k == "coarse_bytes") *value = 8.0 * b->d_Kinv.n;
  else if (k == "n_front_max") *value = std::max(b->bd.maxnf, b->bn.maxnf);
  else if (k == "precision") *value = b->prec;
  else if (k == "n_adaptive") *value = b->n_adaptive;
  else {
    for (auto& pr : b->times)
      if (pr.first == k) {
        *value = pr.second;
        return VEM_OK;
      }
    set_last_error("bddc_info: unknown key " + k);
    return VEM_EINVAL;
  }
  return VEM_OK;
}

extern "C" void bddc_free(bddc* b) { delete b; }

extern "C" int bddc_time_local_solves(bddc* b, int nrep, double* ms, double* bytes) {
  if (!b || nrep <= 0 || !ms || !bytes) { set_last_error("bddc_time_local_solves: bad argument"); return VEM_EINVAL; }
  try {
    const BddcView V = make_view(b);
    cudaStream_t st = b->stream;
    b->XN.zero(st);
    b->XD.zero(st);
    auto sweeps = [&]() {
      if (b->prec == 0) {
        sweep_batch<double>(b, b->bn, V, b->bn.F.p, b->XN.p, b->UVN.p, 1);
        sweep_batch<double>(b, b->bd, V, b->bd.F.p, b->XD.p, b->UVD.p, 1);
      } else {
        sweep_batch<float>(b, b->bn, V, b->bn.F32.p, b->XN.p, b->UVN.p, 1);
        sweep_batch<float>(b, b->bd, V, b->bd.F32.p, b->XD.p, b->UVD.p, 1);
      }
    };
    sweeps();   // warm-up
    cudaEvent_t e0, e1;
    VB_CUDA(cudaEventCreate(&e0));
    VB_CUDA(cudaEventCreate(&e1));
    VB_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < nrep; ++i) sweeps();
    VB_CUDA(cudaEventRecord(e1, st));
    VB_CUDA(cudaEventSynchronize(e1));
    float t = 0;
    VB_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / nrep;
    // algorithmic bytes: every panel read once forward and once backward
    *bytes = 2.0 * (b->prec == 0 ? 8.0 : 4.0) * (double)(b->bn.nF + b->bd.nF);
    return VEM_OK;
  } catch (const Error& e) {
    return bfail(e);
  }
}

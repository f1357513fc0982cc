// vem_system: element construction on the GPU (one CTA per element), the
// deterministic CSR assembly of K = [A B^T; B 0] (Eq. MatrixForm), the load
// (Eq. discreteF) and the operator apply.
#include "system.h"
#include "elem_body.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>

namespace vb {

// element-independent tables: a device copy for the kernels
struct ElemTablesDev;

template <int K>
struct KElement {
  const ElemRec* rec;
  const double* xyz;
  const double* nu;
  const int64_t* offK;
  const int64_t* offK2;
  const ElemTables* tab;
  double *A, *B, *P0, *WM, *scratch;
  size_t stride;
  int nE, nblocks;
  int* status;
  VB_HD void operator()(const KExec& ex, int blk) const {
    ElemShared<K>& sh = *reinterpret_cast<ElemShared<K>*>(ex.smem);
    ElemRec& R = *reinterpret_cast<ElemRec*>(ex.smem + (sizeof(ElemShared<K>) + 7) / 8);
    double* scr = scratch + (size_t)blk * stride;
    for (int e = blk; e < nE; e += nblocks) {
      const int* src = reinterpret_cast<const int*>(rec + e);
      int* dst = reinterpret_cast<int*>(&R);
      for (int i = ex.tid; i < (int)(sizeof(ElemRec) / sizeof(int)); i += ex.nt) dst[i] = src[i];
      ex.sync();
      ElemBuilder<K> b(R, xyz, *tab, sh, scr, ex);
      const int np = pdim3(K - 1);
      bool ok = b.build(nu[e], A + offK2[e], B + (size_t)np * offK[e], P0 + (size_t)3 * pdim3(K) * offK[e],
                        WM + (size_t)np * e);
      if (!ok && ex.tid == 0) flag_error(status, 1);
      ex.sync();
    }
  }
};

// CSR assembly: one CTA per system row; contributions gathered element by
// element in a fixed order (deterministic sums, no atomics).
struct KAssemble {
  int64_t nvf;
  int np;
  const int64_t* rowptr;
  const int* col;
  double* val;
  const int64_t *adj_ptr;
  const int *adj_elem, *adj_loc;
  const int64_t *offK, *offK2, *sysdof;
  const double *A, *B;
  VB_HD void operator()(const KExec& ex, int r) const {
    const int64_t r0 = rowptr[r], r1 = rowptr[r + 1];
    for (int64_t p = r0 + ex.tid; p < r1; p += ex.nt) val[p] = 0.0;
    ex.sync();
    for (int64_t q = adj_ptr[r]; q < adj_ptr[r + 1]; ++q) {
      const int e = adj_elem[q], loc = adj_loc[q];
      const int nK = (int)(offK[e + 1] - offK[e]);
      const int64_t* sd = sysdof + offK[e];
      const double* Ae = A + offK2[e];
      const double* Be = B + (int64_t)np * offK[e];
      const int ncols = loc < nK ? nK + np : nK;
      for (int b = ex.tid; b < ncols; b += ex.nt) {
        int64_t c;
        double v;
        if (loc < nK) {
          if (b < nK) { c = sd[b]; v = Ae[(int64_t)loc * nK + b]; }
          else { c = nvf + (int64_t)e * np + (b - nK); v = Be[(int64_t)(b - nK) * nK + loc]; }
        } else {
          c = sd[b];
          v = Be[(int64_t)(loc - nK) * nK + b];
        }
        if (c < 0) continue;
        int64_t lo = r0, hi = r1 - 1;
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (col[mid] < c) lo = mid + 1; else hi = mid;
        }
        val[lo] += v;
      }
      ex.sync();
    }
  }
};

// y = K x: each CTA handles nt/32 rows, one warp per row
struct KSpmv {
  int64_t nrows;
  const int64_t* rowptr;
  const int* col;
  const double* val;
  const double* x;
  double* y;
  __device__ void operator()(const KExec& ex, int blk) const {
    int lane = ex.tid & 31;
    int64_t r = (int64_t)blk * (ex.nt >> 5) + (ex.tid >> 5);
    if (r >= nrows) return;
    double acc = 0.0;
    for (int64_t p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32) acc += val[p] * __ldg(x + col[p]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = acc;
  }
};

// load-rule points of an element: tetrahedra (x_K, outward fan triangle)
struct LoadRule {
  int nq;
  double x[16], w[16];
};

VB_HD inline void elem_centroid(const ElemRec& R, const double* xyz, double* xK) {
  xK[0] = xK[1] = xK[2] = 0.0;
  for (int i = 0; i < R.nv; ++i)
    for (int d = 0; d < 3; ++d) xK[d] += xyz[3 * R.vert[i] + d];
  for (int d = 0; d < 3; ++d) xK[d] /= R.nv;
}

VB_HD inline void load_point(const LoadRule& L, const ElemRec& R, const double* xyz, const double* xK, int p,
                             double* x, double* w) {
  const int nq = L.nq, nq3 = nq * nq * nq;
  int tet = p / nq3, q = p % nq3;
  int iu = q / (nq * nq), iv = (q / nq) % nq, iw = q % nq;
  int f = 0, t = 0, cnt = 0;
  for (f = 0; f < R.nf; ++f) {
    int nt = R.fnv[f] - 2;
    if (tet < cnt + nt) { t = tet - cnt + 1; break; }
    cnt += nt;
  }
  int m = R.fnv[f];
  int i0 = 0, i1 = t, i2 = t + 1;
  if (R.fsign[f] < 0) { i0 = m - 1; i1 = m - 1 - t; i2 = m - 2 - t; }
  const int* lv = R.floopv[f];
  double a1[3], b1[3], c1[3];
  for (int d = 0; d < 3; ++d) {
    a1[d] = xyz[3 * R.vert[lv[i0]] + d] - xK[d];
    b1[d] = xyz[3 * R.vert[lv[i1]] + d] - xK[d];
    c1[d] = xyz[3 * R.vert[lv[i2]] + d] - xK[d];
  }
  double cr[3];
  cross3(b1, c1, cr);
  double det = a1[0] * cr[0] + a1[1] * cr[1] + a1[2] * cr[2];
  double U = L.x[iu], V = L.x[iv], W = L.x[iw];
  double px = U, py = V * (1 - U), pz = W * (1 - U) * (1 - V);
  *w = L.w[iu] * L.w[iv] * L.w[iw] * (1 - U) * (1 - U) * (1 - V) * det;
  for (int d = 0; d < 3; ++d) x[d] = xK[d] + px * a1[d] + py * b1[d] + pz * c1[d];
}

struct KQuadPoints {
  const ElemRec* rec;
  const double* xyz;
  const int64_t* qoff;
  LoadRule L;
  double* out;
  VB_HD void operator()(const KExec& ex, int e) const {
    const ElemRec& R = rec[e];
    double xK[3];
    elem_centroid(R, xyz, xK);
    int npts = (int)(qoff[e + 1] - qoff[e]);
    for (int p = ex.tid; p < npts; p += ex.nt) {
      double x[3], w;
      load_point(L, R, xyz, xK, p, x, &w);
      for (int d = 0; d < 3; ++d) out[3 * (qoff[e] + p) + d] = x[d];
    }
  }
};

// Tetrahedron `tet` of the element's load rule, (x_K, fan triangle): its
// edge vectors from x_K and the determinant (6 |T|).
VB_HD inline void load_tet(const ElemRec& R, const double* xyz, const double* xK, int tet, double* a1, double* b1,
                           double* c1, double* det) {
  int f = 0, t = 0, cnt = 0;
  for (f = 0; f < R.nf; ++f) {
    int nt = R.fnv[f] - 2;
    if (tet < cnt + nt) { t = tet - cnt + 1; break; }
    cnt += nt;
  }
  int m = R.fnv[f];
  int i0 = 0, i1 = t, i2 = t + 1;
  if (R.fsign[f] < 0) { i0 = m - 1; i1 = m - 1 - t; i2 = m - 2 - t; }
  const int* lv = R.floopv[f];
  for (int d = 0; d < 3; ++d) {
    a1[d] = xyz[3 * R.vert[lv[i0]] + d] - xK[d];
    b1[d] = xyz[3 * R.vert[lv[i1]] + d] - xK[d];
    c1[d] = xyz[3 * R.vert[lv[i2]] + d] - xK[d];
  }
  double cr[3];
  cross3(b1, c1, cr);
  *det = a1[0] * cr[0] + a1[1] * cr[1] + a1[2] * cr[2];
}

// per element: F[c][a] = sum_p w f_c m_a(xi); local rhs = P0^T F (Eq. discreteF).
// k = 2, 3: every thread takes points of the rule (tetrahedron by
// tetrahedron, the tetrahedron geometry once per thread), evaluates the
// monomials once per point and accumulates all 3 dim P_k moments in
// registers; the threads' partial sums are added by a fixed tree.  k = 4
// (105 moments): the load-rule points are generated once each, in chunks
// staged in shared memory (scaled coordinates and w f), and every (c, a)
// moment sums over the chunk in point order.
template <int K>
struct KLoadLocal {
  const ElemRec* rec;
  const double* xyz;
  const int64_t* qoff;
  const double* fq;
  const int64_t* offK;
  const double* P0;
  const ElemTables* tab;
  LoadRule L;
  double* rloc;
  static constexpr int CH = 128;   // points per staged chunk (k = 4)
  static constexpr int NT = 128;   // threads per element
  static constexpr bool PER_THREAD = 3 * pdim3(K) <= 60;
  static size_t smem_bytes() {
    return sizeof(double) * (3 * pdim3(K) + 4 + (PER_THREAD ? (size_t)NT * 3 * pdim3(K) : 6 * CH));
  }
  __device__ void operator()(const KExec& ex, int e) const {
    constexpr int NP1 = pdim3(K);
    double* Fm = ex.smem;
    double* geo = ex.smem + 3 * NP1;   // xK[3], hK
    const ElemRec& R = rec[e];
    if (ex.tid == 0) {
      elem_centroid(R, xyz, geo);
      double h2 = 0;
      for (int i = 0; i < R.nv; ++i)
        for (int j = i + 1; j < R.nv; ++j) {
          double s = 0;
          for (int d = 0; d < 3; ++d) {
            double t = xyz[3 * R.vert[i] + d] - xyz[3 * R.vert[j] + d];
            s += t * t;
          }
          h2 = s > h2 ? s : h2;
        }
      geo[3] = sqrt(h2);
    }
    ex.sync();
    const int npts = (int)(qoff[e + 1] - qoff[e]);
    if constexpr (PER_THREAD) {
      double* part = geo + 4;          // [nt][3 NP1]
      double acc[3 * NP1];
      for (int q = 0; q < 3 * NP1; ++q) acc[q] = 0.0;
      const double xK[3] = {geo[0], geo[1], geo[2]}, hinv = 1.0 / geo[3];
      const int nq = L.nq, nq3 = nq * nq * nq;
      const int ntet = npts / nq3;
      const double* fe = fq + 3 * qoff[e];
      for (int tet = 0; tet < ntet; ++tet) {
        double a1[3], b1[3], c1[3], det;
        load_tet(R, xyz, xK, tet, a1, b1, c1, &det);
        for (int q = ex.tid; q < nq3; q += ex.nt) {
          const int iu = q / (nq * nq), iv = (q / nq) % nq, iw = q % nq;
          const double U = L.x[iu], V = L.x[iv], W = L.x[iw];
          const double px = U, py = V * (1 - U), pz = W * (1 - U) * (1 - V);
          const double w = L.w[iu] * L.w[iv] * L.w[iw] * (1 - U) * (1 - U) * (1 - V) * det;
          double xi[3];
          for (int d = 0; d < 3; ++d) xi[d] = (px * a1[d] + py * b1[d] + pz * c1[d]) * hinv;
          double mono[NP1];
          for (int a = 0; a < NP1; ++a) {
            const Exp3 ea = tab->e3[a];
            mono[a] = ipow(xi[0], ea.a) * ipow(xi[1], ea.b) * ipow(xi[2], ea.c);
          }
          const double* fp = fe + 3 * ((int64_t)tet * nq3 + q);
          for (int c = 0; c < 3; ++c) {
            const double wf = w * fp[c];
            for (int a = 0; a < NP1; ++a) acc[c * NP1 + a] += wf * mono[a];
          }
        }
      }
      for (int q = 0; q < 3 * NP1; ++q) part[(int64_t)ex.tid * 3 * NP1 + q] = acc[q];
      ex.sync();
      for (int st = 1; st < ex.nt; st <<= 1) {
        if ((ex.tid & (2 * st - 1)) == 0 && ex.tid + st < ex.nt)
          for (int q = 0; q < 3 * NP1; ++q)
            part[(int64_t)ex.tid * 3 * NP1 + q] += part[(int64_t)(ex.tid + st) * 3 * NP1 + q];
        ex.sync();
      }
      for (int q = ex.tid; q < 3 * NP1; q += ex.nt) Fm[q] = part[q];
      ex.sync();
    } else {
      double* pt = geo + 4;              // [CH][6]: scaled x, y, z, then w f_c
      const int c = ex.tid / NP1, a = ex.tid % NP1;
      const bool mine = ex.tid < 3 * NP1;
      const Exp3 ea = tab->e3[mine ? a : 0];
      double acc = 0.0;
      for (int p0 = 0; p0 < npts; p0 += CH) {
        const int cnt = npts - p0 < CH ? npts - p0 : CH;
        for (int q = ex.tid; q < cnt; q += ex.nt) {
          double x[3], w;
          load_point(L, R, xyz, geo, p0 + q, x, &w);
          double* d = pt + 6 * q;
          for (int k = 0; k < 3; ++k) d[k] = (x[k] - geo[k]) / geo[3];
          for (int k = 0; k < 3; ++k) d[3 + k] = w * fq[3 * (qoff[e] + p0 + q) + k];
        }
        ex.sync();
        if (mine)
          for (int q = 0; q < cnt; ++q) {
            const double* d = pt + 6 * q;
            acc += d[3 + c] * ipow(d[0], ea.a) * ipow(d[1], ea.b) * ipow(d[2], ea.c);
          }
        ex.sync();
      }
      if (mine) Fm[ex.tid] = acc;
      ex.sync();
    }
    int nK = (int)(offK[e + 1] - offK[e]);
    const double* P = P0 + (size_t)3 * NP1 * offK[e];
    for (int col = ex.tid; col < nK; col += ex.nt) {
      double s = 0.0;
      for (int q = 0; q < 3 * NP1; ++q) s += P[(size_t)q * nK + col] * Fm[q];
      rloc[offK[e] + col] = s;
    }
  }
};

// system rhs from the per-element local vectors (velocity rows), zero pressure rows
struct KGatherRhs {
  int64_t nrows, nvf;
  const int64_t* adj_ptr;
  const int *adj_elem, *adj_loc;
  const int64_t* offK;
  const double* rloc;
  double* rhs;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < nrows ? (int64_t)(blk + 1) * 256 : nrows;
    for (int64_t r = (int64_t)blk * 256 + ex.tid; r < hi; r += ex.nt) {
      double acc = 0.0;
      if (r < nvf)
        for (int64_t q = adj_ptr[r]; q < adj_ptr[r + 1]; ++q) acc += rloc[offK[adj_elem[q]] + adj_loc[q]];
      rhs[r] = acc;
    }
  }
};

// reduced scheme: keep row 0 (the constant-pressure row, the face fluxes) of
// every element's B_K, one CTA per element
struct KCompactB {
  const double* Bfull;
  double* B;
  const int64_t* offK;
  int npf;
  VB_HD void operator()(const KExec& ex, int e) const {
    const int64_t o = offK[e], nK = offK[e + 1] - o;
    for (int64_t c = ex.tid; c < nK; c += ex.nt) B[o + c] = Bfull[(int64_t)npf * o + c];
  }
};

// the element kernel's working buffers and outputs still to be checked: the
// kernel runs while the host builds the CSR pattern, and finish_elements
// reads its status afterwards (the buffers live until then)
struct ElemPending {
  DBuf<double> scratch, wm, Bfull;
  DBuf<int> status;
  int npf = 0;
};

template <int K>
static void launch_elements(vem_system* s, const DBuf<int64_t>& offK, const DBuf<int64_t>& offK2,
                            ElemPending& pe) {
  const int nE = s->topo.nE;
  const int grid = std::min(nE, 152 * (K == 2 ? 8 : (K == 3 ? 4 : 2)));
  size_t stride = ElemScratch<K>::size(s->nKmax);
  pe.scratch.alloc((size_t)grid * stride);
  pe.status.alloc(1);
  pe.status.zero(s->stream);
  size_t smem = ((sizeof(ElemShared<K>) + 7) / 8) * 8 + sizeof(ElemRec);
  pe.npf = pdim3(K - 1);
  pe.wm.alloc((size_t)nE * pe.npf);
  // the reduced scheme keeps one B row per element: the full rows go to a
  // temporary and row 0 is copied out
  double* Bdst = s->d_B.p;
  if (s->dof.reduced) {
    pe.Bfull.alloc((size_t)pe.npf * s->h_eoff.back());
    Bdst = pe.Bfull.p;
  }
  KElement<K> f{s->d_rec.p, s->d_xyz.p, s->d_nu.p, offK.p, offK2.p, s->d_tab.p, s->d_A.p, Bdst,
                s->d_P0.p, pe.wm.p, pe.scratch.p, stride, nE, grid, pe.status.p};
  launch_lb128<4>(f, grid, smem, s->stream);
  if (s->dof.reduced) launch(KCompactB{pe.Bfull.p, s->d_B.p, offK.p, pe.npf}, nE, 128, 0, s->stream);
}

static void finish_elements(vem_system* s, ElemPending& pe) {
  const int nE = s->topo.nE;
  auto st = pe.status.download(s->stream);
  VB_CHECK(st[0] == 0, VEM_ESINGULAR, "element projector system singular (degenerate element)");
  std::vector<double> w = pe.wm.download(s->stream);
  if (s->dof.reduced) {
    s->elem_wmean.assign(nE, 0.0);
    for (int e = 0; e < nE; ++e) s->elem_wmean[e] = w[(size_t)e * pe.npf];
  } else {
    s->elem_wmean = std::move(w);
  }
  pe.scratch.release();
  pe.Bfull.release();
}

static void load_tables(vem_system* s) {
  std::vector<ElemTables> T(1);
  make_elem_tables(s->dof.k, T[0]);
  s->d_tab.upload(T, s->stream);
}

}  // namespace vb

using namespace vb;

static int fail(const Error& e) {
  set_last_error(e.what());
  return e.status;
}

extern "C" const char* vem_last_error(void) { return vb::g_last_error.c_str(); }

static int assemble(const vem_mesh* mesh, int k, const double* nu, bool reduced, vem_system** out) {
  if (!out || !nu) { set_last_error("vem_assemble: null argument"); return VEM_EINVAL; }
  *out = nullptr;
  if (k < 2 || k > 4) { set_last_error("vem_assemble: degree k must be 2, 3 or 4"); return VEM_EINVAL; }
  vem_system* s = new vem_system();
  try {
    auto t0 = std::chrono::steady_clock::now();
    auto mark = [&](const char* name) {
      auto t1 = std::chrono::steady_clock::now();
      s->times.push_back({name, std::chrono::duration<double, std::milli>(t1 - t0).count()});
      t0 = t1;
    };
    build_topology(mesh, s->topo);
    number_dofs(s->topo, k, s->dof, reduced);
    const Topo& t = s->topo;
    const DofNumbering& d = s->dof;
    std::vector<ElemRec> recs;
    build_elem_records(t, d, recs);
    // per-element offsets and system DOF maps
    std::vector<int64_t> offK(t.nE + 1, 0), offK2(t.nE + 1, 0);
    for (int e = 0; e < t.nE; ++e) {
      offK[e + 1] = offK[e] + recs[e].nK;
      offK2[e + 1] = offK2[e] + (int64_t)recs[e].nK * recs[e].nK;
      s->nKmax = std::max(s->nKmax, recs[e].nK);
    }
    s->h_eoff = offK;
    s->h_sysdof.assign(offK[t.nE], -1);
    std::vector<int64_t> g;
    for (int e = 0; e < t.nE; ++e) {
      element_global_dofs(t, d, e, g);
      VB_CHECK((int)g.size() == recs[e].nK, VEM_EINVAL, "element DOF count mismatch");
      for (size_t i = 0; i < g.size(); ++i) s->h_sysdof[offK[e] + i] = d.free_index[g[i]];
    }
    mark("t_topology_ms");
    // upload element data, build element matrices
    s->d_rec.alloc(t.nE);
    VB_CUDA(cudaMemcpyAsync(s->d_rec.p, recs.data(), recs.size() * sizeof(ElemRec), cudaMemcpyHostToDevice, s->stream));
    s->d_xyz.upload(t.xyz, s->stream);
    s->d_nu.upload(std::vector<double>(nu, nu + t.nE), s->stream);
    DBuf<int64_t> dK, dK2;
    dK.upload(offK, s->stream);
    dK2.upload(offK2, s->stream);
    s->d_A.alloc(offK2[t.nE]);
    s->d_B.alloc((size_t)d.np * offK[t.nE]);
    s->d_P0.alloc((size_t)3 * pdim3(k) * offK[t.nE]);
    s->d_sysdof.upload(s->h_sysdof, s->stream);
    load_tables(s);
    ElemPending pe;
    if (k == 2) launch_elements<2>(s, dK, dK2, pe);
    else if (k == 3) launch_elements<3>(s, dK, dK2, pe);
    else launch_elements<4>(s, dK, dK2, pe);
    mark("t_element_launch_ms");
    // CSR pattern and row adjacency (host, overlapping the element kernel)
    const int64_t nvf = d.nvf, np = d.np;
    s->n = nvf + d.npress;
    std::vector<int64_t> cnt(s->n + 1, 0);
    for (int e = 0; e < t.nE; ++e)
      for (int i = 0; i < recs[e].nK; ++i) {
        int64_t r = s->h_sysdof[offK[e] + i];
        if (r >= 0) cnt[r + 1]++;
      }
    for (int64_t r = nvf; r < s->n; ++r) cnt[r + 1] = 1;
    for (int64_t r = 0; r < s->n; ++r) cnt[r + 1] += cnt[r];
    s->h_adj_ptr = cnt;
    s->h_adj_elem.assign(cnt[s->n], 0);
    s->h_adj_loc.assign(cnt[s->n], 0);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int e = 0; e < t.nE; ++e)
      for (int i = 0; i < recs[e].nK; ++i) {
        int64_t r = s->h_sysdof[offK[e] + i];
        if (r >= 0) { s->h_adj_elem[fill[r]] = e; s->h_adj_loc[fill[r]] = i; fill[r]++; }
      }
    for (int e = 0; e < t.nE; ++e)
      for (int a = 0; a < np; ++a) {
        int64_t r = nvf + (int64_t)e * np + a;
        s->h_adj_elem[fill[r]] = e;
        s->h_adj_loc[fill[r]] = recs[e].nK + a;
        fill[r]++;
      }
    std::vector<int64_t> rowptr;
    std::vector<int> cols;
    build_csr_pattern(recs, offK, s->h_sysdof, s->h_adj_ptr, s->h_adj_elem, s->h_adj_loc, nvf, (int)np, s->n,
                      rowptr, cols);
    mark("t_pattern_ms");
    finish_elements(s, pe);
    mark("t_element_wait_ms");
    VB_CHECK(s->n < (int64_t)INT32_MAX, VEM_EINVAL, "system too large for 32-bit column indices");
    s->nnz = rowptr[s->n];
    s->d_rowptr.upload(rowptr, s->stream);
    s->d_col.upload(cols, s->stream);
    s->d_val.alloc(s->nnz);
    s->d_adj_ptr.upload(s->h_adj_ptr, s->stream);
    s->d_adj_elem.upload(s->h_adj_elem, s->stream);
    s->d_adj_loc.upload(s->h_adj_loc, s->stream);
    s->d_eoff.upload(offK, s->stream);
    KAssemble fa{nvf, (int)np, s->d_rowptr.p, s->d_col.p, s->d_val.p, s->d_adj_ptr.p, s->d_adj_elem.p,
                 s->d_adj_loc.p, s->d_eoff.p, dK2.p, s->d_sysdof.p, s->d_A.p, s->d_B.p};
    launch(fa, s->n, 32, 0, s->stream);

    s->d_eoffK2 = std::move(dK2);
    mark("t_pattern_upload_ms");
    VB_CUDA(cudaStreamSynchronize(s->stream));
    mark("t_gpu_finish_ms");
    *out = s;
    return VEM_OK;
  } catch (const Error& e) {
    delete s;
    return fail(e);
  } catch (const std::exception& e) {
    delete s;
    set_last_error(e.what());
    return VEM_ENOMEM;
  }
}

extern "C" int vem_assemble(const vem_mesh* mesh, int k, const double* nu, vem_system** out) {
  return assemble(mesh, k, nu, false, out);
}

extern "C" int vem_assemble_reduced(const vem_mesh* mesh, int k, const double* nu, vem_system** out) {
  return assemble(mesh, k, nu, true, out);
}

extern "C" int vem_info(const vem_system* s, const char* key, double* value) {
  if (!s || !key || !value) { set_last_error("vem_info: null argument"); return VEM_EINVAL; }
  const std::string k(key);
  if (k == "nnz") { *value = (double)s->nnz; return VEM_OK; }
  if (k == "n_elements") { *value = s->topo.nE; return VEM_OK; }
  if (k == "reduced") { *value = s->dof.reduced ? 1.0 : 0.0; return VEM_OK; }
  for (auto& pr : s->times)
    if (pr.first == k) { *value = pr.second; return VEM_OK; }
  set_last_error("vem_info: unknown key " + k);
  return VEM_EINVAL;
}

extern "C" int vem_dof_layout(const vem_system* s, int64_t* nvf, int64_t* np, int64_t* nvel) {
  if (!s) { set_last_error("null system"); return VEM_EINVAL; }
  if (nvf) *nvf = s->dof.nvf;
  if (np) *np = s->dof.npress;
  if (nvel) *nvel = s->dof.nvel;
  return VEM_OK;
}

extern "C" int vem_free_dofs(const vem_system* s, int64_t* out) {
  if (!s || !out) { set_last_error("null argument"); return VEM_EINVAL; }
  std::memcpy(out, s->dof.free_to_global.data(), s->dof.nvf * sizeof(int64_t));
  return VEM_OK;
}

static void load_offsets(vem_system* s, int degree, std::vector<int64_t>& qoff, LoadRule& L) {
  VB_CHECK(degree >= 0 && degree <= 24, VEM_EINVAL, "load degree out of range");
  int nq = (degree + 3) / 2 + 1;
  L = LoadRule{};
  L.nq = nq;
  gauss01(nq, L.x, L.w);
  const Topo& t = s->topo;
  qoff.assign(t.nE + 1, 0);
  for (int e = 0; e < t.nE; ++e) {
    // face loop sizes as in the element records (build_elem_records)
    const int* ef = &t.elem_face[t.elem_ptr[e]];
    const int ntets = elem_fan_tets(t.elem_ptr[e + 1] - t.elem_ptr[e], [&](int fi) {
      const int f = std::abs(ef[fi]) - 1;
      return t.face_ptr[f + 1] - t.face_ptr[f];
    });
    qoff[e + 1] = qoff[e] + (int64_t)ntets * nq * nq * nq;
  }
}

extern "C" int vem_quad_points(vem_system* s, int degree, int64_t* n, double* xyz_out) {
  if (!s || !n) { set_last_error("null argument"); return VEM_EINVAL; }
  try {
    std::vector<int64_t> qoff;
    LoadRule L;
    load_offsets(s, degree, qoff, L);
    *n = qoff.back();
    if (!xyz_out) return VEM_OK;
    DBuf<int64_t> dq;
    dq.upload(qoff, s->stream);
    DBuf<double> pts(3 * (size_t)qoff.back());
    launch(KQuadPoints{s->d_rec.p, s->d_xyz.p, dq.p, L, pts.p}, s->topo.nE, 128, 0, s->stream);
    VB_CUDA(cudaMemcpyAsync(xyz_out, pts.p, pts.n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    VB_CUDA(cudaStreamSynchronize(s->stream));
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

extern "C" int vem_load(vem_system* s, int degree, const double* fq, double* rhs) {
  if (!s || !fq || !rhs) { set_last_error("null argument"); return VEM_EINVAL; }
  try {
    std::vector<int64_t> qoff;
    LoadRule L;
    load_offsets(s, degree, qoff, L);
    DBuf<int64_t> dq;
    dq.upload(qoff, s->stream);
    // f on the device is read in place; host f is copied in
    cudaPointerAttributes pa{};
    const bool on_dev = cudaPointerGetAttributes(&pa, fq) == cudaSuccess &&
                        (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    DBuf<double> df(on_dev ? 0 : 3 * (size_t)qoff.back());
    if (!on_dev)
      VB_CUDA(cudaMemcpyAsync(df.p, fq, df.n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    const double* fsrc = on_dev ? fq : df.p;
    DBuf<double> rloc(s->h_eoff.back());
    const int nE = s->topo.nE;
    if (s->dof.k == 2)
      launch(KLoadLocal<2>{s->d_rec.p, s->d_xyz.p, dq.p, fsrc, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc.p}, nE,
             KLoadLocal<2>::NT, KLoadLocal<2>::smem_bytes(), s->stream);
    else if (s->dof.k == 3)
      launch(KLoadLocal<3>{s->d_rec.p, s->d_xyz.p, dq.p, fsrc, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc.p}, nE,
             KLoadLocal<3>::NT, KLoadLocal<3>::smem_bytes(), s->stream);
    else
      launch(KLoadLocal<4>{s->d_rec.p, s->d_xyz.p, dq.p, fsrc, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc.p}, nE,
             KLoadLocal<4>::NT, KLoadLocal<4>::smem_bytes(), s->stream);
    launch(KGatherRhs{s->n, s->dof.nvf, s->d_adj_ptr.p, s->d_adj_elem.p, s->d_adj_loc.p, s->d_eoff.p, rloc.p, rhs},
           (s->n + 255) / 256, 256, 0, s->stream);
    VB_CUDA(cudaStreamSynchronize(s->stream));
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

namespace vb {
// Non-homogeneous Dirichlet data (test support): per element, the rows of
// [A_e; B_e] applied to the prescribed values of its fixed velocity DOFs.
// One CTA per element.
struct KLiftLocal {
  const int64_t *offK, *offK2, *sysdof, *eglob;
  const double *A, *B, *g;
  int np;
  double* rloc;    // velocity rows, element-local layout
  double* rp;      // pressure rows, e * np + a
  VB_HD void operator()(const KExec& ex, int e) const {
    const int64_t o = offK[e];
    const int nK = (int)(offK[e + 1] - o);
    const double* Ae = A + offK2[e];
    const double* Be = B + (int64_t)np * o;
    for (int a = ex.tid; a < nK + np; a += ex.nt) {
      double acc = 0.0;
      for (int b = 0; b < nK; ++b) {
        if (sysdof[o + b] >= 0) continue;
        const double gb = g[eglob[o + b]];
        acc += (a < nK ? Ae[(int64_t)a * nK + b] : Be[(int64_t)(a - nK) * nK + b]) * gb;
      }
      if (a < nK) rloc[o + a] = acc;
      else rp[(int64_t)e * np + (a - nK)] = acc;
    }
  }
};

// f -= the gathered element rows (velocity rows by the DOF adjacency,
// pressure rows directly)
struct KLiftGather {
  int64_t nrows, nvf;
  const int64_t* adj_ptr;
  const int *adj_elem, *adj_loc;
  const int64_t* offK;
  const double *rloc, *rp;
  double* f;
  VB_HD void operator()(const KExec& ex, int blk) const {
    const int64_t hi = (int64_t)(blk + 1) * 256 < nrows ? (int64_t)(blk + 1) * 256 : nrows;
    for (int64_t r = (int64_t)blk * 256 + ex.tid; r < hi; r += ex.nt) {
      double acc = 0.0;
      if (r < nvf) {
        for (int64_t q = adj_ptr[r]; q < adj_ptr[r + 1]; ++q) acc += rloc[offK[adj_elem[q]] + adj_loc[q]];
      } else {
        acc = rp[r - nvf];
      }
      f[r] -= acc;
    }
  }
};

void spmv(vem_system* s, const double* x, double* y, cudaStream_t st) {
  launch(KSpmv{s->n, s->d_rowptr.p, s->d_col.p, s->d_val.p, x, y}, (s->n + 7) / 8, 256, 0, st);
}
}  // namespace vb

extern "C" int vem_lift_dirichlet(vem_system* s, const double* g_host, double* f_dev) {
  if (!s || !g_host || !f_dev) { set_last_error("vem_lift_dirichlet: null argument"); return VEM_EINVAL; }
  try {
    const Topo& t = s->topo;
    const DofNumbering& d = s->dof;
    std::vector<int64_t> eglob(s->h_eoff.back()), ge;
    for (int e = 0; e < t.nE; ++e) {
      element_global_dofs(t, d, e, ge);
      std::copy(ge.begin(), ge.end(), eglob.begin() + s->h_eoff[e]);
    }
    std::vector<int64_t> offK2(t.nE + 1, 0);
    for (int e = 0; e < t.nE; ++e) {
      const int64_t nK = s->h_eoff[e + 1] - s->h_eoff[e];
      offK2[e + 1] = offK2[e] + nK * nK;
    }
    DBuf<int64_t> dglob, dK2;
    dglob.upload(eglob, s->stream);
    dK2.upload(offK2, s->stream);
    DBuf<double> dg(d.nvel), rloc(s->h_eoff.back()), rp((size_t)d.np * t.nE);
    VB_CUDA(cudaMemcpyAsync(dg.p, g_host, sizeof(double) * d.nvel, cudaMemcpyHostToDevice, s->stream));
    launch(KLiftLocal{s->d_eoff.p, dK2.p, s->d_sysdof.p, dglob.p, s->d_A.p, s->d_B.p, dg.p, d.np, rloc.p, rp.p}, t.nE,
           128, 0, s->stream);
    launch(KLiftGather{s->n, d.nvf, s->d_adj_ptr.p, s->d_adj_elem.p, s->d_adj_loc.p, s->d_eoff.p, rloc.p, rp.p, f_dev},
           (s->n + 255) / 256, 256, 0, s->stream);
    VB_CUDA(cudaStreamSynchronize(s->stream));
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

extern "C" int vem_apply(vem_system* s, const double* x, double* y) {
  if (!s || !x || !y) { set_last_error("null argument"); return VEM_EINVAL; }
  try {
    spmv(s, x, y, s->stream);
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

extern "C" int vem_element_matrices(vem_system* s, const int32_t* elems, int32_t count, int32_t* nKout, double* A,
                                    double* B, int64_t* dofs) {
  if (!s || !elems || !nKout || count <= 0) { set_last_error("bad argument"); return VEM_EINVAL; }
  try {
    const auto& off = s->h_eoff;
    int nK = (int)(off[elems[0] + 1] - off[elems[0]]);
    const int np = s->dof.np;
    std::vector<int64_t> g;
    for (int i = 0; i < count; ++i) {
      int e = elems[i];
      VB_CHECK(e >= 0 && e < s->topo.nE, VEM_EINVAL, "element index out of range");
      VB_CHECK(off[e + 1] - off[e] == nK, VEM_EINVAL, "elements with different DOF counts");
      int64_t o2 = 0;
      // offset of A: prefix sum of nK^2
      for (int q = 0; q < e; ++q) { int64_t a = off[q + 1] - off[q]; o2 += a * a; }
      if (A) VB_CUDA(cudaMemcpyAsync(A + (size_t)i * nK * nK, s->d_A.p + o2, sizeof(double) * nK * nK, cudaMemcpyDeviceToHost, s->stream));
      if (B) VB_CUDA(cudaMemcpyAsync(B + (size_t)i * np * nK, s->d_B.p + (size_t)np * off[e], sizeof(double) * np * nK, cudaMemcpyDeviceToHost, s->stream));
      if (dofs) {
        element_global_dofs(s->topo, s->dof, e, g);
        for (int j = 0; j < nK; ++j) dofs[(size_t)i * nK + j] = g[j];
      }
    }
    VB_CUDA(cudaStreamSynchronize(s->stream));
    *nKout = nK;
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

extern "C" int vem_csr(vem_system* s, int64_t* n, int64_t* nnz, int64_t* row_ptr, int32_t* col, double* vals) {
  if (!s || !n || !nnz) { set_last_error("null argument"); return VEM_EINVAL; }
  *n = s->n;
  *nnz = s->nnz;
  if (!vals) return VEM_OK;
  try {
    VB_CUDA(cudaMemcpyAsync(row_ptr, s->d_rowptr.p, sizeof(int64_t) * (s->n + 1), cudaMemcpyDeviceToHost, s->stream));
    VB_CUDA(cudaMemcpyAsync(col, s->d_col.p, sizeof(int) * s->nnz, cudaMemcpyDeviceToHost, s->stream));
    VB_CUDA(cudaMemcpyAsync(vals, s->d_val.p, sizeof(double) * s->nnz, cudaMemcpyDeviceToHost, s->stream));
    VB_CUDA(cudaStreamSynchronize(s->stream));
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

extern "C" int vem_set_stream(vem_system* s, void* st) {
  if (!s) { set_last_error("null system"); return VEM_EINVAL; }
  s->stream = (cudaStream_t)st;
  return VEM_OK;
}

extern "C" void vem_free(vem_system* s) { delete s; }

// ------------------------------------------------ load without device allocation
//
// vem_load_noalloc: the load vector of vem_load for callers that may not
// allocate device memory.  Its only scratch is the fixed array below; the
// kernels are the ones vem_load launches (element load vectors, then the
// deterministic gather), preceded by one kernel that writes the quadrature
// point offsets into the same array.

namespace vb {

constexpr int64_t kLoadScratchBytes = 16ll << 20;   // 16 MiB per device
constexpr int kLoadScratchDevices = 64;
static __device__ __align__(256) unsigned char g_load_scratch[kLoadScratchBytes];

// Device address of g_load_scratch on the current device, looked up once
// per device (in host code the symbol is only a host-side stand-in).
static unsigned char* load_scratch_address() {
  static std::mutex mu;
  static void* addr[kLoadScratchDevices] = {};
  int dev = -1;
  VB_CUDA(cudaGetDevice(&dev));
  VB_CHECK(dev >= 0 && dev < kLoadScratchDevices, VEM_EINVAL, "vem_load_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_load_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      throw Error(VEM_ECUDA, std::string("vem_load_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    addr[dev] = p;
  }
  return static_cast<unsigned char*>(addr[dev]);
}

// qoff[e] = first load-rule point of element e, qoff[nE] = total: one CTA,
// each thread owns a contiguous run of elements; exclusive scan of the run
// totals in shared memory
struct KLoadOffsets {
  const ElemRec* rec;
  int nE;
  int64_t pts_per_tet;
  int64_t* qoff;
  __device__ int64_t count(int e) const {
    const ElemRec& R = rec[e];
    return (int64_t)elem_fan_tets(R.nf, [&](int f) { return R.fnv[f]; }) * pts_per_tet;
  }
  __device__ void operator()(const KExec& ex, int) const {
    int64_t* run = reinterpret_cast<int64_t*>(ex.smem);
    const int per = (nE + ex.nt - 1) / ex.nt;
    const int lo = min(nE, ex.tid * per), hi = min(nE, lo + per);
    int64_t s = 0;
    for (int e = lo; e < hi; ++e) s += count(e);
    run[ex.tid] = s;
    ex.sync();
    if (ex.tid == 0) {
      int64_t acc = 0;
      for (int t = 0; t < ex.nt; ++t) {
        const int64_t v = run[t];
        run[t] = acc;
        acc += v;
      }
      qoff[nE] = acc;
    }
    ex.sync();
    int64_t acc = run[ex.tid];
    for (int e = lo; e < hi; ++e) {
      qoff[e] = acc;
      acc += count(e);
    }
  }
};

}  // namespace vb

extern "C" int vem_load_noalloc(vem_system* s, int degree, const double* fq, double* rhs) {
  if (!s || !fq || !rhs) { set_last_error("vem_load_noalloc: null argument"); return VEM_EINVAL; }
  try {
    VB_CHECK(degree >= 0 && degree <= 24, VEM_EINVAL, "vem_load_noalloc: load degree out of range");
    const int nE = s->topo.nE;
    const int64_t nloc = s->h_eoff.back();   // sum of the element DOF counts
    const int64_t off_bytes = ((int64_t)(nE + 1) * 8 + 255) / 256 * 256;
    const int64_t need = off_bytes + nloc * 8;
    if (need > kLoadScratchBytes) {
      char msg[200];
      std::snprintf(msg, sizeof msg,
                    "vem_load_noalloc: this mesh needs %lld bytes of scratch, above the fixed %lld; use vem_load",
                    (long long)need, (long long)kLoadScratchBytes);
      set_last_error(msg);
      return VEM_EINVAL;
    }
    unsigned char* base = load_scratch_address();
    int64_t* qoff = reinterpret_cast<int64_t*>(base);
    double* rloc = reinterpret_cast<double*>(base + off_bytes);
    LoadRule L;
    L.nq = (degree + 3) / 2 + 1;
    gauss01(L.nq, L.x, L.w);
    const int64_t nq3 = (int64_t)L.nq * L.nq * L.nq;
    launch(KLoadOffsets{s->d_rec.p, nE, nq3, qoff}, 1, 1024, sizeof(int64_t) * 1024, s->stream);
    if (s->dof.k == 2)
      launch(KLoadLocal<2>{s->d_rec.p, s->d_xyz.p, qoff, fq, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc}, nE,
             KLoadLocal<2>::NT, KLoadLocal<2>::smem_bytes(), s->stream);
    else if (s->dof.k == 3)
      launch(KLoadLocal<3>{s->d_rec.p, s->d_xyz.p, qoff, fq, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc}, nE,
             KLoadLocal<3>::NT, KLoadLocal<3>::smem_bytes(), s->stream);
    else
      launch(KLoadLocal<4>{s->d_rec.p, s->d_xyz.p, qoff, fq, s->d_eoff.p, s->d_P0.p, s->d_tab.p, L, rloc}, nE,
             KLoadLocal<4>::NT, KLoadLocal<4>::smem_bytes(), s->stream);
    launch(KGatherRhs{s->n, s->dof.nvf, s->d_adj_ptr.p, s->d_adj_elem.p, s->d_adj_loc.p, s->d_eoff.p, rloc, rhs},
           (s->n + 255) / 256, 256, 0, s->stream);
    return VEM_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

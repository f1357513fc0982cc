// Host preprocessing: mesh topology, DOF numbering (Sec. 3, D1-D5) and the
// fixed-size element records the element kernel reads.
#include "system.h"
#include "launch.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace vb {

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
void set_last_error(const std::string& m) { g_last_error = m; }

void gauss01(int n, double* x, double* w) {
  // roots of the Legendre polynomial P_n by Newton iteration from the
  // Chebyshev-like first guess; weights 2 / ((1 - z^2) P_n'(z)^2); mapped
  // to (0, 1).  The first guesses, and so the roots, decrease with i: they
  // are stored in reverse for increasing nodes.
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      pp = n * (z * p1 - p0) / (z * z - 1.0);
      double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-15) break;
    }
    // derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    pp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 0.5 * (2.0 / ((1.0 - z * z) * pp * pp));
  }
  for (int i = 1; i < n; ++i) VB_CHECK(x[i] > x[i - 1], VEM_EINVAL, "gauss01: nodes out of order");
}

void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  gauss01(n, x.data(), w.data());
}

std::vector<double> lobatto_interior(int k) {
  // the k-1 roots of P_k' on (-1,1), mapped to (0,1)
  std::vector<double> r;
  if (k == 2) r = {0.5};
  else if (k == 3) r = {0.5 * (1.0 - 1.0 / std::sqrt(5.0)), 0.5 * (1.0 + 1.0 / std::sqrt(5.0))};
  else if (k == 4) r = {0.5 * (1.0 - std::sqrt(3.0 / 7.0)), 0.5, 0.5 * (1.0 + std::sqrt(3.0 / 7.0))};
  else throw Error(VEM_EINVAL, "degree k must be 2, 3 or 4");
  return r;
}

void build_topology(const vem_mesh* m, Topo& t) {
  VB_CHECK(m && m->xyz && m->face_ptr && m->face_vtx && m->elem_ptr && m->elem_face, VEM_EINVAL,
           "vem_mesh has a null array");
  VB_CHECK(m->nV > 0 && m->nF > 0 && m->nE > 0, VEM_EINVAL, "empty mesh");
  t.nV = m->nV;
  t.nF = m->nF;
  t.nE = m->nE;
  t.xyz.assign(m->xyz, m->xyz + 3 * (size_t)m->nV);
  t.face_ptr.assign(m->face_ptr, m->face_ptr + m->nF + 1);
  t.face_vtx.assign(m->face_vtx, m->face_vtx + t.face_ptr[m->nF]);
  t.elem_ptr.assign(m->elem_ptr, m->elem_ptr + m->nE + 1);
  t.elem_face.assign(m->elem_face, m->elem_face + t.elem_ptr[m->nE]);
  for (int f = 0; f < t.nF; ++f) {
    int nv = t.face_ptr[f + 1] - t.face_ptr[f];
    VB_CHECK(nv >= 3 && nv <= kMaxFaceVerts, VEM_EINVAL, "face with unsupported vertex count");
    for (int i = t.face_ptr[f]; i < t.face_ptr[f + 1]; ++i)
      VB_CHECK(t.face_vtx[i] >= 0 && t.face_vtx[i] < t.nV, VEM_EINVAL, "face vertex out of range");
  }
  // edges by first appearance in the face loops
  std::unordered_map<uint64_t, int> eid;
  t.face_edges_ptr.assign(t.nF + 1, 0);
  t.face_edges.clear();
  for (int f = 0; f < t.nF; ++f) {
    int b = t.face_ptr[f], nv = t.face_ptr[f + 1] - b;
    for (int i = 0; i < nv; ++i) {
      int va = t.face_vtx[b + i], vb_ = t.face_vtx[b + (i + 1) % nv];
      int lo = std::min(va, vb_), hi = std::max(va, vb_);
      uint64_t key = ((uint64_t)lo << 32) | (uint32_t)hi;
      auto it = eid.find(key);
      int id;
      if (it == eid.end()) {
        id = (int)t.edge_a.size();
        eid.emplace(key, id);
        t.edge_a.push_back(lo);
        t.edge_b.push_back(hi);
      } else {
        id = it->second;
      }
      t.face_edges.push_back(id);
    }
    t.face_edges_ptr[f + 1] = (int)t.face_edges.size();
  }
  t.nEd = (int)t.edge_a.size();
  std::vector<int> cnt(t.nF, 0);
  for (int e = 0; e < t.nE; ++e)
    for (int i = t.elem_ptr[e]; i < t.elem_ptr[e + 1]; ++i) {
      int s = t.elem_face[i];
      int f = std::abs(s) - 1;
      VB_CHECK(s != 0 && f < t.nF, VEM_EINVAL, "element face reference out of range");
      cnt[f]++;
    }
  t.bnd_f.assign(t.nF, 0);
  t.bnd_v.assign(t.nV, 0);
  t.bnd_e.assign(t.nEd, 0);
  for (int f = 0; f < t.nF; ++f) {
    VB_CHECK(cnt[f] == 1 || cnt[f] == 2, VEM_EINVAL, "face shared by more than two elements or unused");
    if (cnt[f] == 1) {
      t.bnd_f[f] = 1;
      for (int i = t.face_ptr[f]; i < t.face_ptr[f + 1]; ++i) t.bnd_v[t.face_vtx[i]] = 1;
      for (int i = t.face_edges_ptr[f]; i < t.face_edges_ptr[f + 1]; ++i) t.bnd_e[t.face_edges[i]] = 1;
    }
  }
  t.elem_verts.assign(t.nE, {});
  t.elem_edges.assign(t.nE, {});
  for (int e = 0; e < t.nE; ++e) {
    auto& vs = t.elem_verts[e];
    auto& es = t.elem_edges[e];
    for (int i = t.elem_ptr[e]; i < t.elem_ptr[e + 1]; ++i) {
      int f = std::abs(t.elem_face[i]) - 1;
      for (int j = t.face_ptr[f]; j < t.face_ptr[f + 1]; ++j) vs.push_back(t.face_vtx[j]);
      for (int j = t.face_edges_ptr[f]; j < t.face_edges_ptr[f + 1]; ++j) es.push_back(t.face_edges[j]);
    }
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    VB_CHECK((int)vs.size() <= kMaxElemVerts && (int)es.size() <= kMaxElemEdges &&
                 t.elem_ptr[e + 1] - t.elem_ptr[e] <= kMaxElemFaces,
             VEM_EINVAL, "element too large for the element kernel");
  }
}

// reduced: the reduced scheme (the remark after the convergence theorem):
// every D5 DOF (element divergence moment of degree >= 1) is fixed to zero
// like a Dirichlet DOF, and the pressure keeps one constant per element
void number_dofs(const Topo& t, int k, DofNumbering& d, bool reduced) {
  VB_CHECK(k >= 2 && k <= 4, VEM_EINVAL, "degree k must be 2, 3 or 4");
  d.k = k;
  d.ce = 3 * (k - 1);
  d.cf = 3 * pdim2(k - 2);
  d.n4 = n_d4(k);
  d.n5 = n_d5(k);
  d.np_full = pdim3(k - 1);
  d.np = reduced ? 1 : d.np_full;
  d.reduced = reduced;
  d.off_e = 3LL * t.nV;
  d.off_f = d.off_e + (int64_t)t.nEd * d.ce;
  d.off_k = d.off_f + (int64_t)t.nF * d.cf;
  d.nvel = d.off_k + (int64_t)t.nE * (d.n4 + d.n5);
  std::vector<char> fixed(d.nvel, 0);
  for (int v = 0; v < t.nV; ++v)
    if (t.bnd_v[v]) fixed[3 * v] = fixed[3 * v + 1] = fixed[3 * v + 2] = 1;
  for (int e = 0; e < t.nEd; ++e)
    if (t.bnd_e[e]) for (int j = 0; j < d.ce; ++j) fixed[d.off_e + (int64_t)e * d.ce + j] = 1;
  for (int f = 0; f < t.nF; ++f)
    if (t.bnd_f[f]) for (int j = 0; j < d.cf; ++j) fixed[d.off_f + (int64_t)f * d.cf + j] = 1;
  if (reduced)
    for (int e = 0; e < t.nE; ++e)
      for (int j = 0; j < d.n5; ++j) fixed[d.off_k + (int64_t)e * (d.n4 + d.n5) + d.n4 + j] = 1;
  d.free_index.assign(d.nvel, -1);
  d.free_to_global.clear();
  for (int64_t g = 0; g < d.nvel; ++g)
    if (!fixed[g]) {
      d.free_index[g] = (int64_t)d.free_to_global.size();
      d.free_to_global.push_back(g);
    }
  d.nvf = (int64_t)d.free_to_global.size();
  d.npress = (int64_t)t.nE * d.np;
}

void element_global_dofs(const Topo& t, const DofNumbering& d, int e, std::vector<int64_t>& out) {
  out.clear();
  for (int v : t.elem_verts[e]) for (int c = 0; c < 3; ++c) out.push_back(3LL * v + c);
  for (int ed : t.elem_edges[e])
    for (int j = 0; j < d.ce; ++j) out.push_back(d.off_e + (int64_t)ed * d.ce + j);
  for (int i = t.elem_ptr[e]; i < t.elem_ptr[e + 1]; ++i) {
    int f = std::abs(t.elem_face[i]) - 1;
    for (int j = 0; j < d.cf; ++j) out.push_back(d.off_f + (int64_t)f * d.cf + j);
  }
  for (int j = 0; j < d.n4 + d.n5; ++j) out.push_back(d.off_k + (int64_t)e * (d.n4 + d.n5) + j);
}

void build_elem_records(const Topo& t, const DofNumbering& d, std::vector<ElemRec>& recs) {
  recs.assign(t.nE, ElemRec{});
  for (int e = 0; e < t.nE; ++e) {
    ElemRec& r = recs[e];
    const auto& vs = t.elem_verts[e];
    const auto& es = t.elem_edges[e];
    r.nv = (int)vs.size();
    r.ne = (int)es.size();
    r.nf = t.elem_ptr[e + 1] - t.elem_ptr[e];
    for (int i = 0; i < r.nv; ++i) r.vert[i] = vs[i];
    for (int i = 0; i < r.ne; ++i) { r.edge_a[i] = t.edge_a[es[i]]; r.edge_b[i] = t.edge_b[es[i]]; }
    for (int fi = 0; fi < r.nf; ++fi) {
      int s = t.elem_face[t.elem_ptr[e] + fi];
      int f = std::abs(s) - 1;
      r.face[fi] = f;
      r.fsign[fi] = s > 0 ? 1 : -1;
      int b = t.face_ptr[f], nv = t.face_ptr[f + 1] - b;
      r.fnv[fi] = nv;
      for (int i = 0; i < nv; ++i) {
        int va = t.face_vtx[b + i], vbb = t.face_vtx[b + (i + 1) % nv];
        r.floopv[fi][i] = (int)(std::lower_bound(vs.begin(), vs.end(), va) - vs.begin());
        int ed = t.face_edges[t.face_edges_ptr[f] + i];
        r.floope[fi][i] = (int)(std::lower_bound(es.begin(), es.end(), ed) - es.begin());
        r.floopdir[fi][i] = va < vbb ? 1 : 0;
      }
    }
    r.nK = 3 * r.nv + r.ne * d.ce + r.nf * d.cf + d.n4 + d.n5;
  }
}

}  // namespace vb

#include "elem_body.cuh"
namespace vb {

void build_csr_pattern(const std::vector<ElemRec>& recs, const std::vector<int64_t>& offK,
                       const std::vector<int64_t>& sysdof, const std::vector<int64_t>& adj_ptr,
                       const std::vector<int>& adj_elem, const std::vector<int>& adj_loc, int64_t nvf, int np,
                       int64_t n, std::vector<int64_t>& rowptr, std::vector<int>& cols) {
  // Two parallel passes over the rows: count the distinct columns of each
  // row, then write them sorted into their final place.  Each thread marks
  // the columns of its current row in a bitmap (de-duplication without
  // sorting the repeats) and clears the marks afterwards.
  rowptr.assign(n + 1, 0);
  auto row_cols = [&](int64_t r, std::vector<uint64_t>& bits, std::vector<int>& buf) {
    buf.clear();
    for (int64_t q = adj_ptr[r]; q < adj_ptr[r + 1]; ++q) {
      const int e = adj_elem[q], loc = adj_loc[q];
      const int nK = recs[e].nK;
      for (int bb = 0; bb < nK; ++bb) {
        const int64_t cc = sysdof[offK[e] + bb];
        if (cc < 0) continue;
        uint64_t& w = bits[cc >> 6];
        const uint64_t m = (uint64_t)1 << (cc & 63);
        if (!(w & m)) {
          w |= m;
          buf.push_back((int)cc);
        }
      }
      if (loc < nK)   // a velocity row: the element's pressures (distinct per element)
        for (int a = 0; a < np; ++a) buf.push_back((int)(nvf + (int64_t)e * np + a));
    }
    for (int x : buf)
      if (x < nvf) bits[x >> 6] = 0;   // every marked bit belongs to this row
  };
#pragma omp parallel
  {
    std::vector<uint64_t> bits((size_t)((n + 63) / 64), 0);
    std::vector<int> buf;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t r = 0; r < n; ++r) {
      row_cols(r, bits, buf);
      rowptr[r + 1] = (int64_t)buf.size();
    }
#pragma omp single
    {
      for (int64_t r = 0; r < n; ++r) rowptr[r + 1] += rowptr[r];
      cols.resize(rowptr[n]);
    }
#pragma omp for schedule(dynamic, 1024)
    for (int64_t r = 0; r < n; ++r) {
      row_cols(r, bits, buf);
      std::sort(buf.begin(), buf.end());
      std::copy(buf.begin(), buf.end(), cols.begin() + rowptr[r]);
    }
  }
}



void make_elem_tables(int k, ElemTables& T) {
  T = ElemTables{};
  int i = 0;
  for (int d = 0; i < kMaxMono3; ++d)
    for (int a = d; a >= 0 && i < kMaxMono3; --a)
      for (int b = d - a; b >= 0 && i < kMaxMono3; --b) {
        T.e3[i] = Exp3{(unsigned char)a, (unsigned char)b, (unsigned char)(d - a - b), (unsigned char)d};
        ++i;
      }
  i = 0;
  for (int d = 0; i < kMaxMono2; ++d)
    for (int a = d; a >= 0 && i < kMaxMono2; --a) {
      T.e2[i] = Exp2{(unsigned char)a, (unsigned char)(d - a), (unsigned char)d, 0};
      ++i;
    }
  std::vector<double> gl = lobatto_interior(k);
  for (size_t j = 0; j < gl.size(); ++j) T.gl[j] = gl[j];
  std::vector<double> x, w;
  // edges: exact to degree 2k+3
  T.nq_edge = k + 2;
  gauss01(T.nq_edge, x, w);
  for (int j = 0; j < T.nq_edge; ++j) { T.qe_x[j] = x[j]; T.qe_w[j] = w[j]; }
  // faces: collapsed triangle rule exact to degree 2k+2
  T.nq_face = (2 * k + 5) / 2;
  gauss01(T.nq_face, x, w);
  for (int j = 0; j < T.nq_face; ++j) { T.qf_x[j] = x[j]; T.qf_w[j] = w[j]; }
  // volume: collapsed tetrahedron rule exact to degree 2k
  T.nq_vol = k + 2;
  gauss01(T.nq_vol, x, w);
  for (int j = 0; j < T.nq_vol; ++j) { T.qv_x[j] = x[j]; T.qv_w[j] = w[j]; }
}

}  // namespace vb

extern "C" int vem_kernel_launches(int64_t* count) {
  if (!count) return VEM_EINVAL;
  *count = vb::g_launches.load();
  return VEM_OK;
}

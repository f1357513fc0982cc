// Host-side BDDC setup (Sec. 4-6): interface classification into macro
// vertices, edges and faces, the primal constraints of Sec. 5.1 as a
// Householder change of basis, and the nested-dissection symbolic analysis
// of the subdomain Dirichlet, constrained Neumann and deluxe face (and edge)
// problems.
#include "bddc_setup.h"

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <numeric>

namespace vb {

namespace {

struct UF {
  std::vector<int> p;
  explicit UF(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int a) {
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
  }
  void unite(int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

// entity of a global velocity DOF: type (0 vertex, 1 edge, 2 face, 3 element) and id
inline void dof_entity(const DofNumbering& d, int64_t g, int& type, int64_t& id) {
  if (g < d.off_e) { type = 0; id = g / 3; }
  else if (g < d.off_f) { type = 1; id = (g - d.off_e) / d.ce; }
  else if (g < d.off_k) { type = 2; id = (g - d.off_f) / d.cf; }
  else { type = 3; id = (g - d.off_k) / (d.n4 + d.n5); }
}

void face_frame(const Topo& t, int f, double* n, double* t1, double* t2, double& area) {
  int b = t.face_ptr[f], m = t.face_ptr[f + 1] - b;
  double nn[3] = {0, 0, 0};
  for (int i = 0; i < m; ++i) {
    const double* a = &t.xyz[3 * t.face_vtx[b + i]];
    const double* c = &t.xyz[3 * t.face_vtx[b + (i + 1) % m]];
    nn[0] += a[1] * c[2] - a[2] * c[1];
    nn[1] += a[2] * c[0] - a[0] * c[2];
    nn[2] += a[0] * c[1] - a[1] * c[0];
  }
  double ln = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
  area = 0.5 * ln;
  for (int q = 0; q < 3; ++q) n[q] = nn[q] / ln;
  const double* p0 = &t.xyz[3 * t.face_vtx[b]];
  const double* p1 = &t.xyz[3 * t.face_vtx[b + 1]];
  double d[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
  double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
  double lt = 0;
  for (int q = 0; q < 3; ++q) { d[q] -= dn * n[q]; lt += d[q] * d[q]; }
  lt = std::sqrt(lt);
  for (int q = 0; q < 3; ++q) t1[q] = d[q] / lt;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// Area centroid of face f (fan triangles from loop vertex 0).
static void face_centroid(const Topo& t, int f, double* c) {
  int b = t.face_ptr[f], m = t.face_ptr[f + 1] - b;
  const double* p0 = &t.xyz[3 * t.face_vtx[b]];
  double acc[3] = {0, 0, 0}, at = 0;
  for (int i = 1; i < m - 1; ++i) {
    const double* p1 = &t.xyz[3 * t.face_vtx[b + i]];
    const double* p2 = &t.xyz[3 * t.face_vtx[b + i + 1]];
    double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double v[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
    double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double a = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int q = 0; q < 3; ++q) acc[q] += a * (p0[q] + p1[q] + p2[q]) / 3.0;
    at += a;
  }
  for (int q = 0; q < 3; ++q) c[q] = acc[q] / at;
}

// Smallest over largest eigenvalue of a symmetric 6 x 6 matrix (cyclic Jacobi).
static double eig_ratio6(double G[6][6]) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 6; ++q) off += G[p][q] * G[p][q];
    if (off < 1e-300) break;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 6; ++q) {
        if (G[p][q] == 0.0) continue;
        double th = 0.5 * (G[q][q] - G[p][p]) / G[p][q];
        double tt = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        double c = 1.0 / std::sqrt(tt * tt + 1.0), sn = tt * c;
        for (int r = 0; r < 6; ++r) {
          double a = G[r][p], b = G[r][q];
          G[r][p] = c * a - sn * b;
          G[r][q] = sn * a + c * b;
        }
        for (int r = 0; r < 6; ++r) {
          double a = G[p][r], b = G[q][r];
          G[p][r] = c * a - sn * b;
          G[q][r] = sn * a + c * b;
        }
      }
  }
  double lo = G[0][0], hi = G[0][0];
  for (int p = 1; p < 6; ++p) { lo = std::min(lo, G[p][p]); hi = std::max(hi, G[p][p]); }
  return hi > 0 ? lo / hi : 0.0;
}

// Sec. 5.1 (the recipe that satisfies the assumption on the coarse space):
// the primal constraints of a subdomain must control its rigid body modes,
// checked numerically.  For every floating subdomain (no Dirichlet DOF) the
// vertex, edge and face constraints it takes part in are evaluated on the
// six rigid body modes (translations, and rotations about its centroid
// scaled by its diameter); fewer than six independent values leave the
// local Neumann problem singular: VEM_ESINGULAR.  Adaptive rows only add
// constraints and are not needed for the check.
static void check_rigid_modes(const vem_system* s, const int32_t* part, const SetupOptions& o, const BddcHost& H) {
  const Topo& t = s->topo;
  const DofNumbering& d = s->dof;
  const int N = H.N;
  std::vector<char> floating(N, 1);
  for (int e = 0; e < t.nE; ++e)
    for (int64_t q = s->h_eoff[e]; q < s->h_eoff[e + 1]; ++q)
      if (s->h_sysdof[q] < 0) floating[part[e]] = 0;
  const std::vector<double> gl = lobatto_interior(d.k);
  // position of a nodal DOF (vertex or edge node); false for other DOFs
  auto node_pos = [&](int64_t g, double* x, int& comp) {
    if (g < d.off_e) {
      const int v = (int)(g / 3);
      comp = (int)(g % 3);
      for (int q = 0; q < 3; ++q) x[q] = t.xyz[3 * v + q];
      return true;
    }
    if (g < d.off_f) {
      const int64_t r = g - d.off_e;
      const int ed = (int)(r / d.ce), j = (int)((r % d.ce) / 3);
      comp = (int)(r % 3);
      const double* a = &t.xyz[3 * t.edge_a[ed]];
      const double* b = &t.xyz[3 * t.edge_b[ed]];
      for (int q = 0; q < 3; ++q) x[q] = a[q] + gl[j] * (b[q] - a[q]);
      return true;
    }
    return false;
  };
  for (int i = 0; i < N; ++i) {
    if (!floating[i]) continue;
    // centroid and diameter (bounding box) of the subdomain's vertices
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, cen[3] = {0, 0, 0};
    int nvx = 0;
    for (int e : H.subs[i].elems)
      for (int v : t.elem_verts[e]) {
        for (int q = 0; q < 3; ++q) {
          lo[q] = std::min(lo[q], t.xyz[3 * v + q]);
          hi[q] = std::max(hi[q], t.xyz[3 * v + q]);
          cen[q] += t.xyz[3 * v + q];
        }
        ++nvx;
      }
    double Hd = 0;
    for (int q = 0; q < 3; ++q) { cen[q] /= nvx; Hd = std::max(Hd, hi[q] - lo[q]); }
    // rigid mode l at x, component c
    auto rigid = [&](int l, const double* x, int c) {
      if (l < 3) return c == l ? 1.0 : 0.0;
      const double y[3] = {(x[0] - cen[0]) / Hd, (x[1] - cen[1]) / Hd, (x[2] - cen[2]) / Hd};
      const int a = l - 3;                       // e_a x y
      const double cr[3] = {a == 1 ? y[2] * 1.0 : (a == 2 ? -y[1] : 0.0),
                            a == 2 ? y[0] : (a == 0 ? -y[2] : 0.0),
                            a == 0 ? y[1] : (a == 1 ? -y[0] : 0.0)};
      return cr[c];
    };
    std::vector<std::array<double, 6>> rows;
    for (size_t gi = 0; gi < H.macros.size(); ++gi) {
      const Macro& G = H.macros[gi];
      if (!std::binary_search(G.share.begin(), G.share.end(), i)) continue;
      if (G.kind == 0) {
        if (!(o.constraints & 1)) continue;
        for (int64_t r : G.dofs) {
          double x[3];
          int c;
          if (!node_pos(d.free_to_global[r], x, c)) continue;
          std::array<double, 6> row;
          for (int l = 0; l < 6; ++l) row[l] = rigid(l, x, c);
          rows.push_back(row);
        }
      } else if (G.kind == 1) {
        if (!(o.constraints & 2)) continue;
        for (int c = 0; c < 3; ++c) {
          std::array<double, 6> row{};
          int cnt = 0;
          for (int64_t r : G.dofs) {
            double x[3];
            int cc;
            if (!node_pos(d.free_to_global[r], x, cc) || cc != c) continue;
            for (int l = 0; l < 6; ++l) row[l] += rigid(l, x, c);
            ++cnt;
          }
          for (auto& v : row) v /= std::max(cnt, 1);
          rows.push_back(row);
        }
      } else {
        // faces: component means sum_f |f| v(x_f) and the normal flux
        std::array<double, 6> comp[3] = {}, flux{};
        std::vector<int> fs;
        for (int64_t r : G.dofs) {
          int ty;
          int64_t id;
          dof_entity(d, d.free_to_global[r], ty, id);
          if (ty == 2 && (d.free_to_global[r] - d.off_f) % d.cf == 0) fs.push_back((int)id);
        }
        for (int f : fs) {
          double nrm[3], t1[3], t2[3], area, xc[3];
          face_frame(t, f, nrm, t1, t2, area);
          face_centroid(t, f, xc);
          // orientation: outward from the first sharing subdomain, as in the flux constraint
          const int64_t fr = d.free_index[d.off_f + (int64_t)f * d.cf];
          int sgn = 0;
          for (int64_t q = s->h_adj_ptr[fr]; q < s->h_adj_ptr[fr + 1]; ++q) {
            const int e = s->h_adj_elem[q];
            if (part[e] != G.share[0]) continue;
            for (int fi = t.elem_ptr[e]; fi < t.elem_ptr[e + 1]; ++fi)
              if (std::abs(t.elem_face[fi]) - 1 == f) sgn = t.elem_face[fi] > 0 ? 1 : -1;
          }
          for (int l = 0; l < 6; ++l) {
            double fl = 0;
            for (int c = 0; c < 3; ++c) {
              comp[c][l] += area * rigid(l, xc, c);
              fl += nrm[c] * rigid(l, xc, c);
            }
            flux[l] += sgn * area * fl;
          }
        }
        if (o.constraints & 4)
          for (int c = 0; c < 3; ++c) rows.push_back(comp[c]);
        if (o.constraints & 8) rows.push_back(flux);
      }
    }
    double Gm[6][6] = {};
    for (auto& r : rows) {
      double nr = 0;
      for (double v : r) nr += v * v;
      if (nr == 0) continue;
      for (int p = 0; p < 6; ++p)
        for (int q = 0; q < 6; ++q) Gm[p][q] += r[p] * r[q] / nr;
    }
    const double ratio = eig_ratio6(Gm);
    if (!(ratio > 1e-14)) {
      char msg[240];
      std::snprintf(msg, sizeof msg,
                    "subdomain %d touches no Dirichlet boundary and its primal constraints do not control its "
                    "rigid body modes (eigenvalue ratio %.1e): its local Neumann problem is singular",
                    i, ratio);
      throw Error(VEM_ESINGULAR, msg);
    }
  }
}

// Householder QR with rank detection of the n x m column-major matrix A
// (columns = constraint functionals); keeps the reflectors of the
// independent columns.
void householder(int n, int m, std::vector<double> A, Macro& G, double tol) {
  G.r = 0;
  G.hv.clear();
  G.tau.clear();
  std::vector<double> norm0(m);
  for (int j = 0; j < m; ++j) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += A[(size_t)j * n + i] * A[(size_t)j * n + i];
    norm0[j] = std::sqrt(s);
  }
  for (int j = 0; j < m && G.r < n; ++j) {
    double* a = &A[(size_t)j * n];
    // apply previous reflectors
    for (int q = 0; q < G.r; ++q) {
      const double* v = &G.hv[(size_t)q * n];
      double dot = 0;
      for (int i = 0; i < n; ++i) dot += v[i] * a[i];
      dot *= G.tau[q];
      for (int i = 0; i < n; ++i) a[i] -= dot * v[i];
    }
    int r = G.r;
    double s = 0;
    for (int i = r; i < n; ++i) s += a[i] * a[i];
    double nx = std::sqrt(s);
    if (nx <= tol * norm0[j] || nx == 0.0) continue;   // dependent functional
    double alpha = a[r] >= 0 ? -nx : nx;
    std::vector<double> v(n, 0.0);
    for (int i = r; i < n; ++i) v[i] = a[i];
    v[r] -= alpha;
    double vv = 0;
    for (int i = r; i < n; ++i) vv += v[i] * v[i];
    G.hv.insert(G.hv.end(), v.begin(), v.end());
    G.tau.push_back(2.0 / vv);
    G.r++;
  }
}

}  // namespace

void hh_apply_T(const Macro& G, const double* v, double* c) {
  const int n = (int)G.dofs.size();
  for (int i = 0; i < n; ++i) c[i] = v[i];
  for (int q = 0; q < G.r && !G.hv.empty(); ++q) {
    const double* h = &G.hv[(size_t)q * n];
    double dot = 0;
    for (int i = 0; i < n; ++i) dot += h[i] * c[i];
    dot *= G.tau[q];
    for (int i = 0; i < n; ++i) c[i] -= dot * h[i];
  }
}

void hh_apply(const Macro& G, const double* c, double* v) {
  const int n = (int)G.dofs.size();
  for (int i = 0; i < n; ++i) v[i] = c[i];
  for (int q = (G.hv.empty() ? 0 : G.r) - 1; q >= 0; --q) {
    const double* h = &G.hv[(size_t)q * n];
    double dot = 0;
    for (int i = 0; i < n; ++i) dot += h[i] * v[i];
    dot *= G.tau[q];
    for (int i = 0; i < n; ++i) v[i] -= dot * h[i];
  }
}

namespace {

struct ETree {
  std::vector<int> order;                  // local elements in tree order
  std::vector<int> lo, hi, left, right, parent;   // per node: range in order, children
  std::vector<int> post;                   // postorder node ids
  std::vector<int> leaf_of;                // local element -> leaf node
  int root = 0;
};

void build_etree(const std::vector<std::array<double, 3>>& cen, int leaf, ETree& T) {
  int ne = (int)cen.size();
  T.order.resize(ne);
  std::iota(T.order.begin(), T.order.end(), 0);
  T.leaf_of.assign(ne, -1);
  std::vector<std::pair<int, int>> stack;
  // iterative recursion: create node, split
  struct Item { int node; };
  T.lo.clear(); T.hi.clear(); T.left.clear(); T.right.clear(); T.parent.clear();
  auto newnode = [&](int l, int h, int par) {
    T.lo.push_back(l); T.hi.push_back(h); T.left.push_back(-1); T.right.push_back(-1); T.parent.push_back(par);
    return (int)T.lo.size() - 1;
  };
  T.root = newnode(0, ne, -1);
  std::vector<int> todo = {T.root};
  while (!todo.empty()) {
    int nd = todo.back();
    todo.pop_back();
    int l = T.lo[nd], h = T.hi[nd];
    if (h - l <= leaf) {
      for (int i = l; i < h; ++i) T.leaf_of[T.order[i]] = nd;
      continue;
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int i = l; i < h; ++i)
      for (int q = 0; q < 3; ++q) {
        mn[q] = std::min(mn[q], cen[T.order[i]][q]);
        mx[q] = std::max(mx[q], cen[T.order[i]][q]);
      }
    int ax = 0;
    for (int q = 1; q < 3; ++q)
      if (mx[q] - mn[q] > mx[ax] - mn[ax] + 1e-12) ax = q;
    int mid = (l + h) / 2;
    std::stable_sort(T.order.begin() + l, T.order.begin() + h, [&](int a, int b) {
      if (cen[a][ax] != cen[b][ax]) return cen[a][ax] < cen[b][ax];
      return a < b;
    });
    int a = newnode(l, mid, nd), b = newnode(mid, h, nd);
    T.left[nd] = a;
    T.right[nd] = b;
    todo.push_back(a);
    todo.push_back(b);
  }
  // postorder
  T.post.clear();
  std::vector<std::pair<int, int>> st = {{T.root, 0}};
  while (!st.empty()) {
    auto& [nd, state] = st.back();
    if (T.left[nd] < 0 || state == 2) {
      T.post.push_back(nd);
      st.pop_back();
      continue;
    }
    int child = state == 0 ? T.left[nd] : T.right[nd];
    state++;
    st.push_back({child, 0});
  }
}

int lca_of(const ETree& T, const std::vector<int>& pos_in_order, const std::vector<int>& elems) {
  int mn = 1 << 30, mx = -1;
  for (int le : elems) {
    mn = std::min(mn, pos_in_order[le]);
    mx = std::max(mx, pos_in_order[le]);
  }
  int nd = T.leaf_of[T.order[mn]];
  while (!(T.lo[nd] <= mn && mx < T.hi[nd])) nd = T.parent[nd];
  return nd;
}

}  // namespace

void bddc_host_setup(const vem_system* s, const int32_t* part, const SetupOptions& o, BddcHost& H,
                     const std::vector<double>& elem_wmean) {
  const Topo& t = s->topo;
  const DofNumbering& d = s->dof;
  const int nE = t.nE;
  const int np = d.np;
  const int64_t nvf = d.nvf;
  H.times.clear();
  auto t0 = std::chrono::steady_clock::now();
  auto mark = [&](const char* name) {
    const auto t1 = std::chrono::steady_clock::now();
    H.times.push_back({name, std::chrono::duration<double, std::milli>(t1 - t0).count()});
    t0 = t1;
  };
  H.part.assign(part, part + nE);
  int N = 0;
  for (int e = 0; e < nE; ++e) {
    VB_CHECK(part[e] >= 0, VEM_EINVAL, "negative subdomain id");
    N = std::max(N, part[e] + 1);
  }
  H.N = N;
  H.subs.assign(N, Subdomain{});
  for (int e = 0; e < nE; ++e) H.subs[part[e]].elems.push_back(e);
  for (int i = 0; i < N; ++i) VB_CHECK(!H.subs[i].elems.empty(), VEM_EINVAL, "empty subdomain id");
  // multiplicity and sharing sets of free velocity DOFs
  H.mult.assign(nvf, 0);
  std::vector<std::vector<int>> share(nvf);
#pragma omp parallel for schedule(static, 4096)
  for (int64_t r = 0; r < nvf; ++r) {
    auto& sv = share[r];
    for (int64_t q = s->h_adj_ptr[r]; q < s->h_adj_ptr[r + 1]; ++q) sv.push_back(part[s->h_adj_elem[q]]);
    std::sort(sv.begin(), sv.end());
    sv.erase(std::unique(sv.begin(), sv.end()), sv.end());
    H.mult[r] = (int)sv.size();
  }
  mark("t_sym_share_ms");
  // ---- macro entities: interface mesh entities grouped by sharing set and connectivity
  // entity (type, id) -> interface entity number, through one flat table
  // over vertices, edges, faces and elements
  const int64_t ent_off[5] = {0, t.nV, (int64_t)t.nV + t.nEd, (int64_t)t.nV + t.nEd + t.nF,
                              (int64_t)t.nV + t.nEd + t.nF + t.nE};
  std::vector<int> ent_index(ent_off[4], -1);
  std::vector<std::pair<int, int64_t>> ents;
  std::vector<std::vector<int64_t>> ent_dofs;
  for (int64_t r = 0; r < nvf; ++r) {
    if (H.mult[r] < 2) continue;
    int ty;
    int64_t id;
    dof_entity(d, d.free_to_global[r], ty, id);
    int& slot = ent_index[ent_off[ty] + id];
    if (slot < 0) {
      slot = (int)ents.size();
      ents.push_back({ty, id});
      ent_dofs.push_back({});
    }
    ent_dofs[slot].push_back(r);
  }
  const int nent = (int)ents.size();
  UF uf(nent);
  auto same = [&](int a, int b) { return share[ent_dofs[a][0]] == share[ent_dofs[b][0]]; };
  auto find_ent = [&](int ty, int64_t id) { return ent_index[ent_off[ty] + id]; };
  for (int ei = 0; ei < nent; ++ei) {
    auto [ty, id] = ents[ei];
    if (ty == 1) {
      for (int v : {t.edge_a[id], t.edge_b[id]}) {
        int o2 = find_ent(0, v);
        if (o2 >= 0 && same(ei, o2)) uf.unite(ei, o2);
      }
    } else if (ty == 2) {
      for (int q = t.face_edges_ptr[id]; q < t.face_edges_ptr[id + 1]; ++q) {
        int o2 = find_ent(1, t.face_edges[q]);
        if (o2 >= 0 && same(ei, o2)) uf.unite(ei, o2);
      }
      for (int q = t.face_ptr[id]; q < t.face_ptr[id + 1]; ++q) {
        int o2 = find_ent(0, t.face_vtx[q]);
        if (o2 >= 0 && same(ei, o2)) uf.unite(ei, o2);
      }
    }
  }
  std::map<int, std::vector<int>> comps;
  for (int ei = 0; ei < nent; ++ei) comps[uf.find(ei)].push_back(ei);
  H.macros.clear();
  for (auto& [root, members] : comps) {
    Macro G;
    G.share = share[ent_dofs[members[0]][0]];
    bool single_vertex = members.size() == 1 && ents[members[0]].first == 0;
    G.kind = single_vertex ? 0 : (G.share.size() == 2 ? 2 : 1);
    for (int ei : members) G.dofs.insert(G.dofs.end(), ent_dofs[ei].begin(), ent_dofs[ei].end());
    std::sort(G.dofs.begin(), G.dofs.end());
    const int n = (int)G.dofs.size();
    // constraint functionals (columns of A = C^T)
    std::vector<double> A;
    int m = 0;
    bool all = (o.constraints & 16) != 0;
    if (all || G.kind == 0) {
      G.r = (all || (o.constraints & 1)) ? n : 0;   // every DOF primal, identity basis
    } else if (G.kind == 1) {
      if (o.constraints & 2) {
        for (int c = 0; c < 3; ++c) {
          std::vector<double> col(n, 0.0);
          int cnt = 0;
          for (int a = 0; a < n; ++a) {
            int64_t g = d.free_to_global[G.dofs[a]];
            int comp = g < d.off_e ? (int)(g % 3) : (int)((g - d.off_e) % 3);
            if (comp == c) { col[a] = 1.0; cnt++; }
          }
          for (auto& x : col) x /= std::max(cnt, 1);
          A.insert(A.end(), col.begin(), col.end());
          m++;
        }
      }
      householder(n, m, A, G, 1e-10);
    } else {
      std::vector<double> comp[3] = {std::vector<double>(n, 0.0), std::vector<double>(n, 0.0),
                                     std::vector<double>(n, 0.0)};
      std::vector<double> flux(n, 0.0);
      int i0 = G.share[0];
      for (int ei : members) {
        if (ents[ei].first != 2) continue;
        int f = (int)ents[ei].second;
        double nrm[3], t1[3], t2[3], area;
        face_frame(t, f, nrm, t1, t2, area);
        int64_t base = d.off_f + (int64_t)f * d.cf;
        int pn = (int)(std::lower_bound(G.dofs.begin(), G.dofs.end(), d.free_index[base]) - G.dofs.begin());
        // the three beta = 0 moments (n, t1, t2) are consecutive free DOFs
        for (int c = 0; c < 3; ++c) {
          comp[c][pn] += area * nrm[c];
          comp[c][pn + 1] += area * t1[c];
          comp[c][pn + 2] += area * t2[c];
        }
        // orientation: outward from the first sharing subdomain
        int sgn = 0;
        for (int64_t q = s->h_adj_ptr[d.free_index[base]]; q < s->h_adj_ptr[d.free_index[base] + 1]; ++q) {
          int e = s->h_adj_elem[q];
          if (part[e] != i0) continue;
          for (int fi = t.elem_ptr[e]; fi < t.elem_ptr[e + 1]; ++fi)
            if (std::abs(t.elem_face[fi]) - 1 == f) sgn = t.elem_face[fi] > 0 ? 1 : -1;
        }
        VB_CHECK(sgn != 0, VEM_EINVAL, "macro face orientation not found");
        flux[pn] += sgn * area;
      }
      if (o.constraints & 4)
        for (int c = 0; c < 3; ++c) { A.insert(A.end(), comp[c].begin(), comp[c].end()); m++; }
      if (o.constraints & 8) { A.insert(A.end(), flux.begin(), flux.end()); m++; }
      const size_t gi = H.macros.size();
      if (gi < o.extra.size() && !o.extra[gi].empty()) {
        VB_CHECK(o.extra[gi].size() % (size_t)n == 0, VEM_EINVAL, "adaptive rows do not match the macro face");
        A.insert(A.end(), o.extra[gi].begin(), o.extra[gi].end());
        m += (int)(o.extra[gi].size() / n);
      }
      householder(n, m, A, G, 1e-10);
    }
    H.macros.push_back(std::move(G));
  }
  mark("t_sym_macros_ms");
  if (!(o.constraints & 16)) check_rigid_modes(s, part, o, H);
  mark("t_sym_rigid_ms");
  // coarse numbering
  int64_t cc = 0;
  for (auto& G : H.macros) {
    G.coarse0 = cc;
    cc += G.r;
  }
  H.ncoarse_vel = cc;
  H.ncoarse = cc + N;
  // ---- subdomain DOF data
  std::vector<int> face_nb_ptr, face_nb;   // element -> face neighbours
  {
    std::vector<std::vector<int>> fe(t.nF);
    for (int e = 0; e < nE; ++e)
      for (int q = t.elem_ptr[e]; q < t.elem_ptr[e + 1]; ++q) fe[std::abs(t.elem_face[q]) - 1].push_back(e);
    std::vector<std::vector<int>> nb(nE);
    for (auto& v : fe)
      if (v.size() == 2) { nb[v[0]].push_back(v[1]); nb[v[1]].push_back(v[0]); }
    face_nb_ptr.assign(nE + 1, 0);
    for (int e = 0; e < nE; ++e) face_nb_ptr[e + 1] = face_nb_ptr[e] + (int)nb[e].size();
    for (auto& v : nb) face_nb.insert(face_nb.end(), v.begin(), v.end());
  }
  std::vector<std::vector<int>> sub_macros(N);
  for (int gi = 0; gi < (int)H.macros.size(); ++gi)
    for (int i : H.macros[gi].share) sub_macros[i].push_back(gi);

  mark("t_sym_neighbours_ms");
  const bool all_primal = (o.constraints & 16) != 0;
  H.probs.clear();
  std::vector<std::vector<Problem>> sub_probs(N);
  std::vector<std::string> errors(N);

#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < N; ++i) {
    try {
      Subdomain& S = H.subs[i];
      const int ne = (int)S.elems.size();
      std::vector<int64_t> vd;
      for (int e : S.elems)
        for (int64_t q = s->h_eoff[e]; q < s->h_eoff[e + 1]; ++q)
          if (s->h_sysdof[q] >= 0) vd.push_back(s->h_sysdof[q]);
      std::sort(vd.begin(), vd.end());
      vd.erase(std::unique(vd.begin(), vd.end()), vd.end());
      S.vdof = vd;
      const int nv = (int)vd.size();
      auto lv = [&](int64_t g) {
        auto it = std::lower_bound(S.vdof.begin(), S.vdof.end(), g);
        return (it != S.vdof.end() && *it == g) ? (int)(it - S.vdof.begin()) : -1;
      };
      std::vector<std::vector<std::pair<int, int>>> adj(nv);
      for (int le = 0; le < ne; ++le) {
        int e = S.elems[le];
        int nK = (int)(s->h_eoff[e + 1] - s->h_eoff[e]);
        for (int b = 0; b < nK; ++b) {
          int64_t g = s->h_sysdof[s->h_eoff[e] + b];
          if (g >= 0) adj[lv(g)].push_back({le, b});
        }
      }
      S.vadj_ptr.assign(nv + 1, 0);
      S.vadj.clear();
      for (int v = 0; v < nv; ++v) {
        for (auto& pr : adj[v]) { S.vadj.push_back(pr.first); S.vadj.push_back(pr.second); }
        S.vadj_ptr[v + 1] = (int)S.vadj.size() / 2;
      }
      S.press.clear();
      S.wmean.clear();
      S.volume = 0;
      for (int e : S.elems)
        for (int a = 0; a < np; ++a) {
          S.press.push_back(nvf + (int64_t)e * np + a);
          S.wmean.push_back(elem_wmean[(size_t)e * np + a]);
          if (a == 0) S.volume += elem_wmean[(size_t)e * np];
        }
      S.macros = sub_macros[i];
      S.iface_vdof.clear();
      for (int v = 0; v < nv; ++v)
        if (H.mult[S.vdof[v]] >= 2) S.iface_vdof.push_back(v);
      // local primal coordinates and constraint rows (multipliers for edges/faces)
      S.coarse.clear();
      std::vector<std::vector<std::pair<int, double>>> vcon(nv);
      int nmult = 0;
      std::vector<char> vertex_primal(nv, 0);
      for (int gi : S.macros) {
        const Macro& G = H.macros[gi];
        const int n = (int)G.dofs.size();
        if (G.r == n && G.hv.empty()) {
          // identity basis: every DOF primal, removed from the Neumann problem
          for (int a = 0; a < n; ++a) {
            S.coarse.push_back(G.coarse0 + a);
            vertex_primal[lv(G.dofs[a])] = 1;
          }
          continue;
        }
        std::vector<double> e(n), col(n);
        for (int q = 0; q < G.r; ++q) {
          std::fill(e.begin(), e.end(), 0.0);
          e[q] = 1.0;
          hh_apply(G, e.data(), col.data());      // primal functional q = (H e_q)^T v
          for (int a = 0; a < n; ++a)
            if (col[a] != 0.0) vcon[lv(G.dofs[a])].push_back({nmult, col[a]});
          S.coarse.push_back(G.coarse0 + q);
          nmult++;
        }
      }
      S.coarse.push_back(H.ncoarse_vel + i);   // p_0
      S.vcon_ptr.assign(nv + 1, 0);
      S.vcon_id.clear();
      S.vcon_coef.clear();
      for (int v = 0; v < nv; ++v) {
        for (auto& pr : vcon[v]) { S.vcon_id.push_back(pr.first); S.vcon_coef.push_back(pr.second); }
        S.vcon_ptr[v + 1] = (int)S.vcon_id.size();
      }
      // nested-dissection element tree
      std::vector<std::array<double, 3>> cen(ne);
      for (int le = 0; le < ne; ++le) {
        int e = S.elems[le];
        std::array<double, 3> c = {0, 0, 0};
        for (int v : t.elem_verts[e])
          for (int q = 0; q < 3; ++q) c[q] += t.xyz[3 * v + q];
        for (int q = 0; q < 3; ++q) c[q] /= t.elem_verts[e].size();
        cen[le] = c;
      }
      ETree T;
      build_etree(cen, o.leaf, T);
      const int nnodes = (int)T.lo.size();
      std::vector<int> pos_in_order(ne);
      for (int q = 0; q < ne; ++q) pos_in_order[T.order[q]] = q;
      std::vector<int> local_of(nE, -1);
      for (int le = 0; le < ne; ++le) local_of[S.elems[le]] = le;
      // pressure constants: survivors (one per connected component of each subtree)
      std::vector<int> const_node(ne, -1);    // node where (le,0) is eliminated; -1: dropped (p*)
      std::vector<std::vector<int>> surv(nnodes);
      for (int nd : T.post) {
        std::vector<int> cand;
        if (T.left[nd] < 0) {
          for (int q = T.lo[nd]; q < T.hi[nd]; ++q) cand.push_back(T.order[q]);
        } else {
          cand = surv[T.left[nd]];
          cand.insert(cand.end(), surv[T.right[nd]].begin(), surv[T.right[nd]].end());
        }
        // components of the node's element set
        int cnt = T.hi[nd] - T.lo[nd];
        std::vector<int> ids(cnt);
        for (int q = 0; q < cnt; ++q) ids[q] = T.order[T.lo[nd] + q];
        std::vector<int> slot(ne, -1);
        for (int q = 0; q < cnt; ++q) slot[ids[q]] = q;
        UF cu(cnt);
        for (int q = 0; q < cnt; ++q) {
          int e = S.elems[ids[q]];
          for (int z = face_nb_ptr[e]; z < face_nb_ptr[e + 1]; ++z) {
            int o2 = local_of[face_nb[z]];
            if (o2 >= 0 && slot[o2] >= 0) cu.unite(q, slot[o2]);
          }
        }
        std::map<int, int> keep;   // component root -> survivor (smallest global element id)
        for (int le : cand) {
          int rt = cu.find(slot[le]);
          auto it = keep.find(rt);
          if (it == keep.end() || S.elems[le] < S.elems[it->second]) keep[rt] = le;
        }
        for (int le : cand) {
          int rt = cu.find(slot[le]);
          if (keep[rt] != le) const_node[le] = nd;
        }
        for (auto& [rt, le] : keep) surv[nd].push_back(le);
        std::sort(surv[nd].begin(), surv[nd].end());
      }
      VB_CHECK(surv[T.root].size() == 1, VEM_EINVAL, "subdomain is not face-connected");
      S.pstar = surv[T.root][0];
      // velocity DOF -> node (LCA of the leaves of its elements)
      std::vector<int> vnode(nv);
      for (int v = 0; v < nv; ++v) {
        std::vector<int> els;
        for (int q = S.vadj_ptr[v]; q < S.vadj_ptr[v + 1]; ++q) els.push_back(S.vadj[2 * q]);
        vnode[v] = lca_of(T, pos_in_order, els);
      }
      // element column -> local velocity DOF (-1: fixed), shared by the problems
      std::vector<int> elv_off(ne + 1, 0), elv;
      for (int le = 0; le < ne; ++le) {
        const int e = S.elems[le];
        for (int64_t q = s->h_eoff[e]; q < s->h_eoff[e + 1]; ++q) {
          const int64_t g = s->h_sysdof[q];
          elv.push_back(g >= 0 ? lv(g) : -1);
        }
        elv_off[le + 1] = (int)elv.size();
      }
      // ---- problems
      std::vector<int> kinds = {PK_DIRICHLET, PK_NEUMANN};
      // deluxe: every macro face, and every macro edge with scaling 2, that
      // has dual coordinates; one problem per subdomain holds all of them
      // (Dirichlet pivots, the entities' DOFs at the root, entity by entity)
      std::vector<int> dl_macro;
      if (o.scaling >= 1 && !all_primal)
        for (int gi : S.macros) {
          const Macro& M = H.macros[gi];
          const bool dlx = M.kind == 2 || (M.kind == 1 && o.scaling == 2);
          if (dlx && M.r < (int)M.dofs.size()) dl_macro.push_back(gi);
        }
      if (!dl_macro.empty()) kinds.push_back(PK_DELUXE);
      for (int kind : kinds) {
        Problem P;
        P.sub = i;
        P.kind = kind;
        P.macro = -1;
        if (kind == PK_DELUXE) P.dl_macros = dl_macro;
        // pivots per node
        std::vector<std::vector<int>> vel_at(nnodes), prs_at(nnodes);
        for (int v = 0; v < nv; ++v) {
          bool iface = H.mult[S.vdof[v]] >= 2;
          bool active;
          if (kind == PK_NEUMANN) active = !vertex_primal[v];
          else active = !iface;
          if (active) vel_at[vnode[v]].push_back(v);
        }
        for (int le = 0; le < ne; ++le)
          for (int a = 0; a < np; ++a) {
            int nd;
            if (a > 0) nd = T.leaf_of[le];
            else nd = const_node[le];
            if (nd >= 0) prs_at[nd].push_back(le * np + a);
          }
        const int nm = kind == PK_NEUMANN ? nmult : 0;
        // positions in postorder
        P.pos_of_vdof.assign(nv, -1);
        std::vector<int> ppos(ne * np, -1);
        std::vector<int> node_of_prob_node;   // problem node -> etree node
        int pos = 0;
        P.nodes.clear();
        std::vector<int> pnode_of_tnode(nnodes, -1);
        for (int nd : T.post) {
          Node Nd;
          Nd.p0 = pos;
          auto& vl = vel_at[nd];
          std::sort(vl.begin(), vl.end());
          for (int v : vl) {
            P.pos_of_vdof[v] = pos++;
            P.dtype.push_back(DT_VEL);
            P.dsrc.push_back(v);
          }
          auto& pl = prs_at[nd];
          std::sort(pl.begin(), pl.end(), [&](int a, int b) {
            int64_t ga = S.press[a], gb = S.press[b];
            return ga < gb;
          });
          for (int pq : pl) {
            ppos[pq] = pos++;
            P.dtype.push_back(DT_PRESS);
            P.dsrc.push_back(pq);
          }
          if (nd == T.root && nm > 0) {
            P.mult0 = pos;
            P.nmult = nm;
            for (int m = 0; m < nm; ++m) {
              pos++;
              P.dtype.push_back(DT_MULT);
              P.dsrc.push_back(m);
            }
          }
          Nd.np = pos - Nd.p0;
          pnode_of_tnode[nd] = (int)P.nodes.size();
          node_of_prob_node.push_back(nd);
          P.nodes.push_back(Nd);
        }
        P.npiv = pos;
        P.bgrp.assign(pos, -1);
        for (size_t t = 0; t < P.dl_macros.size(); ++t) {
          P.dl_b0.push_back(pos - P.npiv);
          for (int64_t g : H.macros[P.dl_macros[t]].dofs) {
            int v = lv(g);
            P.pos_of_vdof[v] = pos++;
            P.dtype.push_back(DT_BORDER);
            P.dsrc.push_back(v);
            P.bgrp.push_back((int)t);
          }
        }
        P.n = pos;
        // element column -> position
        P.elpos_off.assign(ne + 1, 0);
        P.elpos.clear();
        P.elpos.reserve(elv.size() + (size_t)ne * np);
        for (int le = 0; le < ne; ++le) {
          for (int q = elv_off[le]; q < elv_off[le + 1]; ++q)
            P.elpos.push_back(elv[q] >= 0 ? P.pos_of_vdof[elv[q]] : -1);
          for (int a = 0; a < np; ++a) P.elpos.push_back(ppos[le * np + a]);
          P.elpos_off[le + 1] = (int)P.elpos.size();
        }
        // tree links
        for (int pn = 0; pn < (int)P.nodes.size(); ++pn) {
          int nd = node_of_prob_node[pn];
          P.nodes[pn].parent = T.parent[nd] >= 0 ? pnode_of_tnode[T.parent[nd]] : -1;
        }
        P.children.clear();
        for (int pn = 0; pn < (int)P.nodes.size(); ++pn) {
          int nd = node_of_prob_node[pn];
          P.nodes[pn].first_child = (int)P.children.size();
          P.nodes[pn].nchild = 0;
          if (T.left[nd] >= 0) {
            P.children.push_back(pnode_of_tnode[T.left[nd]]);
            P.children.push_back(pnode_of_tnode[T.right[nd]]);
            P.nodes[pn].nchild = 2;
          }
        }
        // borders (postorder: children first): the positions beyond the
        // node's pivots coupled to them, i.e. the children's borders plus the
        // positions of every element touching a pivot (all of them through a
        // velocity pivot, the velocity ones through a pressure pivot) and the
        // constraint multipliers of the velocity pivots; elements and
        // positions are de-duplicated with per-node stamps
        std::vector<std::vector<int>> bset(P.nodes.size());
        std::vector<int> pstamp(P.n, -1), estamp(ne, -1), evstamp(ne, -1), elist, evlist;
        for (int pn = 0; pn < (int)P.nodes.size(); ++pn) {
          Node& Nd = P.nodes[pn];
          const int last = Nd.p0 + Nd.np;
          std::vector<int> cand;
          auto add = [&](int x) {
            if (x >= last && pstamp[x] != pn) {
              pstamp[x] = pn;
              cand.push_back(x);
            }
          };
          for (int c = 0; c < Nd.nchild; ++c)
            for (int x : bset[P.children[Nd.first_child + c]]) add(x);
          elist.clear();
          evlist.clear();
          for (int p = Nd.p0; p < last; ++p) {
            if (P.dtype[p] == DT_VEL) {
              int v = (int)P.dsrc[p];
              for (int q = S.vadj_ptr[v]; q < S.vadj_ptr[v + 1]; ++q) {
                int le = S.vadj[2 * q];
                if (estamp[le] != pn) { estamp[le] = pn; elist.push_back(le); }
              }
              if (kind == PK_NEUMANN)
                for (int q = S.vcon_ptr[v]; q < S.vcon_ptr[v + 1]; ++q) add(P.mult0 + S.vcon_id[q]);
            } else if (P.dtype[p] == DT_PRESS) {
              int le = (int)P.dsrc[p] / np;
              if (evstamp[le] != pn) { evstamp[le] = pn; evlist.push_back(le); }
            }
          }
          for (int le : elist)
            for (int z = P.elpos_off[le]; z < P.elpos_off[le + 1]; ++z) add(P.elpos[z]);
          for (int le : evlist) {
            if (estamp[le] == pn) continue;   // all its positions are in already
            int e = S.elems[le];
            int nK = (int)(s->h_eoff[e + 1] - s->h_eoff[e]);
            for (int b = 0; b < nK; ++b) add(P.elpos[P.elpos_off[le] + b]);
          }
          std::sort(cand.begin(), cand.end());
          bset[pn] = std::move(cand);
          Nd.nb = (int)bset[pn].size();
        }
        // offsets, rel maps, heights
        int64_t panel = 0, upd = 0, uv = 0;
        P.border.clear();
        for (int pn = 0; pn < (int)P.nodes.size(); ++pn) {
          Node& Nd = P.nodes[pn];
          Nd.border_off = (int64_t)P.border.size();
          P.border.insert(P.border.end(), bset[pn].begin(), bset[pn].end());
          int64_t nf = Nd.np + Nd.nb;
          Nd.panel_off = panel;
          panel += nf * Nd.np;
          Nd.upd_off = upd;
          upd += (int64_t)Nd.nb * Nd.nb;
          Nd.uvec_off = uv;
          uv += Nd.nb;
          Nd.height = 0;
          for (int c = 0; c < Nd.nchild; ++c)
            Nd.height = std::max(Nd.height, P.nodes[P.children[Nd.first_child + c]].height + 1);
        }
        P.rel.clear();
        for (int pn = 0; pn < (int)P.nodes.size(); ++pn) {
          Node& Nd = P.nodes[pn];
          Nd.rel_off = (int64_t)P.rel.size();
          if (Nd.parent < 0) {
            continue;
          }
          const Node& Pa = P.nodes[Nd.parent];
          const int* pb = &P.border[Pa.border_off];
          // both borders are sorted: one merge walk
          int q = 0;
          for (int x : bset[pn]) {
            int fi;
            if (x < Pa.p0 + Pa.np) {
              VB_CHECK(x >= Pa.p0, VEM_EINVAL, "symbolic: border entry below the parent's pivots");
              fi = x - Pa.p0;
            } else {
              while (q < Pa.nb && pb[q] < x) ++q;
              VB_CHECK(q < Pa.nb && pb[q] == x, VEM_EINVAL, "symbolic: child border not in parent front");
              fi = Pa.np + q;
            }
            P.rel.push_back(fi);
          }
        }
        if (kind == PK_DELUXE) {
          Node& R = P.nodes.back();
          VB_CHECK(R.nb == P.n - P.npiv, VEM_EINVAL, "symbolic: deluxe root border differs from the entities' DOFs");
          R.flags = 1;
        } else {
          VB_CHECK(P.nodes.back().nb == 0, VEM_EINVAL, "symbolic: root with a border");
        }
        sub_probs[i].push_back(std::move(P));
      }
    } catch (const Error& e) {
      errors[i] = e.what();
    }
  }
  mark("t_sym_subdomains_ms");
  for (int i = 0; i < N; ++i) VB_CHECK(errors[i].empty(), VEM_EINVAL, errors[i]);
  H.dir_prob.assign(N, -1);
  H.neu_prob.assign(N, -1);
  for (int i = 0; i < N; ++i)
    for (auto& P : sub_probs[i]) {
      if (P.kind == PK_DIRICHLET) H.dir_prob[i] = (int)H.probs.size();
      if (P.kind == PK_NEUMANN) H.neu_prob[i] = (int)H.probs.size();
      H.probs.push_back(std::move(P));
    }
  mark("t_sym_collect_ms");
}

}  // namespace vb

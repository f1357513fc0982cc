// Host-side description of a discretized problem (topology, DOF numbering,
// element tables, CSR pattern) and the device objects built from it.
#pragma once
#include "common.h"

namespace vb {

constexpr int kMaxElemVerts = 40;
constexpr int kMaxElemEdges = 64;
constexpr int kMaxElemFaces = 28;
constexpr int kMaxFaceVerts = 12;

// Per-element tables consumed by the element kernel (fixed-size records).
struct ElemRec {
  int nv, ne, nf, nK;
  int vert[kMaxElemVerts];                 // global vertex ids, increasing
  int edge_a[kMaxElemEdges], edge_b[kMaxElemEdges];   // endpoints (a < b), edges by increasing id
  int face[kMaxElemFaces];                 // global face id (element order)
  int fsign[kMaxElemFaces];                // +1: global normal points out of the element
  int fnv[kMaxElemFaces];                  // vertices of the face loop
  int floopv[kMaxElemFaces][kMaxFaceVerts];   // local vertex index of loop vertex i
  int floope[kMaxElemFaces][kMaxFaceVerts];   // local edge index of loop edge (i, i+1)
  int floopdir[kMaxElemFaces][kMaxFaceVerts]; // 1 if loop edge runs from lower to higher vertex id
};

struct Topo {
  int nV = 0, nF = 0, nE = 0, nEd = 0;
  std::vector<double> xyz;
  std::vector<int> face_ptr, face_vtx;
  std::vector<int> elem_ptr, elem_face;
  std::vector<int> edge_a, edge_b;                 // endpoints per edge, a < b
  std::vector<int> face_edges_ptr, face_edges;     // edges of each face loop (loop order)
  std::vector<char> bnd_v, bnd_e, bnd_f;
  std::vector<std::vector<int>> elem_verts, elem_edges;
};

struct DofNumbering {
  int k = 2;
  int ce = 0, cf = 0, n4 = 0, n5 = 0, np = 0;      // per entity / element counts
  int np_full = 0;                                 // dim P_{k-1} (np is 1 in the reduced scheme)
  bool reduced = false;                            // D5 fixed to zero, element-constant pressure
  int64_t off_e = 0, off_f = 0, off_k = 0, nvel = 0;
  int64_t nvf = 0, npress = 0;                     // free velocity, pressures
  std::vector<int64_t> free_index;                 // global velocity -> free index or -1
  std::vector<int64_t> free_to_global;
};

void build_topology(const vem_mesh* m, Topo& t);
void number_dofs(const Topo& t, int k, DofNumbering& d, bool reduced = false);
// element-local velocity DOFs (global numbers) in the element-local order
void element_global_dofs(const Topo& t, const DofNumbering& d, int e, std::vector<int64_t>& out);
void build_elem_records(const Topo& t, const DofNumbering& d, std::vector<ElemRec>& recs);

// Tetrahedra of an element's load rule: (x_K, fan triangle) for every fan
// triangle of every face; one definition for the host point count
// (vem_quad_points, vem_load) and the device offsets (vem_load_noalloc).
template <class FaceVerts>
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int elem_fan_tets(int nf, FaceVerts fnv) {
  int nt = 0;
  for (int f = 0; f < nf; ++f) nt += fnv(f) - 2;
  return nt;
}
// CSR pattern of K = [A B^T; B 0] over the system layout (free velocity,
// then element pressures): row r holds the columns of every element
// adjacent to r (velocity rows also the element's pressures); sorted rows
void build_csr_pattern(const std::vector<ElemRec>& recs, const std::vector<int64_t>& offK,
                       const std::vector<int64_t>& sysdof, const std::vector<int64_t>& adj_ptr,
                       const std::vector<int>& adj_elem, const std::vector<int>& adj_loc, int64_t nvf, int np,
                       int64_t n, std::vector<int64_t>& rowptr, std::vector<int>& cols);

}  // namespace vb

namespace vb { struct ElemTables; }
struct vem_system {
  vb::Topo topo;
  vb::DofNumbering dof;
  cudaStream_t stream = 0;
  std::vector<std::pair<std::string, double>> times;   // vem_assemble phase wall times (ms)
  int nKmax = 0;
  // element tables and outputs on the device
  vb::DBuf<vb::ElemRec> d_rec;
  vb::DBuf<double> d_xyz;
  vb::DBuf<double> d_nu;
  vb::DBuf<vb::ElemTables> d_tab;
  std::vector<double> elem_wmean;   // int_K m_a per element pressure (a in P_{k-1})
  vb::DBuf<int64_t> d_eoff;      // prefix sums of nK (element DOF offsets)
  vb::DBuf<int64_t> d_eoffK2;    // prefix sums of nK^2 (element matrix offsets)
  vb::DBuf<double> d_A;          // element stiffness A_K (nK x nK), concatenated
  vb::DBuf<double> d_B;          // element divergence B_K (np x nK)
  vb::DBuf<double> d_P0;         // Pi^0_k (3 dim P_k x nK) for the load
  vb::DBuf<int64_t> d_sysdof;    // element DOF -> system index (-1 fixed), [sum nK]
  std::vector<int64_t> h_eoff, h_sysdof;   // host copies of the DOF maps
  // global CSR of K (system layout)
  int64_t n = 0, nnz = 0;
  vb::DBuf<int64_t> d_rowptr;
  vb::DBuf<int> d_col;
  vb::DBuf<double> d_val;
  // row -> (element, local index) adjacency for deterministic gathers
  vb::DBuf<int64_t> d_adj_ptr;
  vb::DBuf<int> d_adj_elem, d_adj_loc;
  std::vector<int64_t> h_adj_ptr;
  std::vector<int> h_adj_elem, h_adj_loc;
};

namespace vb {
struct ElemTables;
void make_elem_tables(int k, ElemTables& T);
}

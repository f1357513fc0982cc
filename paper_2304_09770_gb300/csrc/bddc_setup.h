// Host-side BDDC setup data (Sec. 4-6): subdomain DOF sets, macro entities,
// primal constraints with their change of basis, and the symbolic
// (nested-dissection, multifrontal) analysis of every local problem.
#pragma once
#include "system.h"

#include <string>
#include <utility>
#include <vector>

namespace vb {

enum ProbKind { PK_DIRICHLET = 0, PK_NEUMANN = 1, PK_DELUXE = 2 };
enum DofType { DT_VEL = 0, DT_PRESS = 1, DT_MULT = 2, DT_BORDER = 3 };

// Macro entity of the interface (Sec. 5.1): vertex, edge or face, with its
// primal constraints as an implicit orthogonal change of basis: the r
// Householder reflectors H = H_1..H_r of the constraint span; coordinates
// c = H^T v, the first r are primal, the remaining n - r are dual.
struct Macro {
  int kind;                      // 0 vertex, 1 edge, 2 face
  std::vector<int> share;        // sorted subdomain ids
  std::vector<int64_t> dofs;     // system indices (free velocity), increasing
  int r = 0;                     // rank of the primal constraints
  std::vector<double> hv;        // Householder vectors, column-major n x r
  std::vector<double> tau;       // r
  int64_t coarse0 = 0;           // first coarse index of the primal coordinates
};

struct Node {
  int p0 = 0, np = 0, nb = 0;    // pivot range in the problem, border size
  int parent = -1, height = 0;
  int64_t border_off = 0;        // into Problem::border (positions)
  int64_t panel_off = 0;         // into the factor store
  int64_t upd_off = 0;           // into the update-matrix store
  int64_t rel_off = 0;           // child border -> parent front index map (this node as child)
  int64_t uvec_off = 0;          // update vector offset for the solves (per rhs)
  int first_child = 0, nchild = 0;   // into Problem::children
  int flags = 0;                 // 1: assemble border-border entries (deluxe root)
};

struct Problem {
  int sub = 0, kind = 0, macro = -1;
  // deluxe problem of a subdomain: its deluxe entities (macro ids), the
  // first root-border index of each (their DOFs follow one another at the
  // root, entity by entity), and per position the entity's index in
  // dl_macros for those border positions (-1 for the pivots)
  std::vector<int> dl_macros, dl_b0, bgrp;
  int n = 0, npiv = 0;           // positions (pivots first, then border-only)
  int mult0 = 0, nmult = 0;      // multiplier positions [mult0, mult0 + nmult)
  std::vector<int> dtype;        // per position
  std::vector<int64_t> dsrc;     // per position: vel -> local vdof; press -> le*np + a; mult -> id
  std::vector<int> elpos;        // [local elem][nK_e + np] -> position or -1
  std::vector<int> elpos_off;    // per local element
  std::vector<int> pos_of_vdof;  // local vdof -> position or -1
  std::vector<Node> nodes;       // postorder
  std::vector<int> border;       // concatenated border lists
  std::vector<int> children;     // concatenated child node ids (problem-local)
  std::vector<int> rel;          // concatenated rel maps
};

struct Subdomain {
  std::vector<int> elems;              // global element ids
  std::vector<int64_t> vdof;           // system indices of its free velocity DOFs (increasing)
  std::vector<int> vadj_ptr, vadj;     // local vdof -> (local elem, element column) pairs
  std::vector<int> vcon_ptr;           // local vdof -> constraint rows touching it
  std::vector<int> vcon_id;
  std::vector<double> vcon_coef;
  std::vector<int64_t> press;          // system indices of its pressures
  int pstar = -1;                      // local element whose constant pressure is dropped
  double volume = 0.0;
  std::vector<double> wmean;           // int_K m_a for its pressures (local order)
  std::vector<int> macros;             // macro entities it touches
  std::vector<int64_t> coarse;         // local primal coordinate -> coarse index (last: p_0)
  std::vector<int> iface_vdof;         // local vdofs on the interface (increasing)
};

struct BddcHost {
  int N = 0;
  std::vector<int> part;
  std::vector<Subdomain> subs;
  std::vector<Macro> macros;
  std::vector<int> mult;               // per free velocity DOF
  int64_t ncoarse_vel = 0, ncoarse = 0;
  std::vector<Problem> probs;          // Dirichlet(i), Neumann(i), deluxe(i, F)
  std::vector<int> dir_prob, neu_prob; // per subdomain
  std::vector<std::pair<std::string, double>> times;   // host phase times (ms)
};

struct SetupOptions {
  uint32_t constraints = 0xF;    // 1 vertex, 2 edge, 4 face, 8 flux; 16 all-interface-primal
  int scaling = 1;               // 0 multiplicity, 1 deluxe on faces, 2 deluxe on faces and edges
  int leaf = 4;                  // elements per nested-dissection leaf
  // adaptive primal rows (Sec. 6) per macro index: concatenated functionals
  // over the macro's DOFs (its dofs order), appended to the face constraints
  std::vector<std::vector<double>> extra;
};

void bddc_host_setup(const vem_system* s, const int32_t* part, const SetupOptions& o, BddcHost& H,
                     const std::vector<double>& elem_wmean);

// Householder helpers on one entity block (column-major reflectors)
void hh_apply_T(const Macro& G, const double* v, double* c);   // c = H^T v
void hh_apply(const Macro& G, const double* c, double* v);     // v = H c

}  // namespace vb

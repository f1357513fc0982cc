// Device-side records of the BDDC data (flattened over all subdomains and
// local problems).
#pragma once
#include "common.h"

namespace vb {

struct NodeDev {
  int prob, p0, np, nb, parent, height, first_child, nchild, flags, ld;
  int64_t border_off, panel_off, upd_off, rel_off, uvec_off;
};

struct ProbDev {
  int sub, kind, n, npiv, mult0, nmult, root, macro;
  int64_t pos_off;     // dtype / dsrc
  int64_t elpos_off;   // element column -> position table
  int64_t elptr_off;   // per local element offsets into that table
  int64_t pv_off;      // local vdof -> position
  int64_t vec_off;     // problem vector offset (per right-hand side: n entries)
};

struct SubDev {
  int ne, nv, npress, pstar, niface, ncl;   // ncl: local primal coordinates (incl. p_0)
  int dir, neu;
  double volume, wsum;
  int64_t elem_off, vdof_off, vadj_ptr_off, vadj_off, vcon_ptr_off, vcon_off;
  int64_t press_off, iface_off, coarse_off, phi_off, elloc_off, ellocptr_off, loc_off;
  int64_t mcon_ptr_off, mcon_off;
};

struct MacroDev {
  int kind, n, r, nshare, ndual;
  int64_t dofs_off, hv_off, tau_off, coarse0, dual_off, share_off, gpos_off, gif_off, deluxe_off;
  int64_t deluxe_e_off;   // deluxe edge: D^(share[s]) at deluxe_e + deluxe_e_off + s ndual^2; -1 otherwise
};

// the arrays every BDDC kernel reads
struct BddcView {
  // vem system
  int np, k;
  int64_t nvf, n;
  const int64_t *offK, *offK2;
  const double *A, *B;
  const float2* A2;    // A as FP32 (high, low) pairs for the refinement residual, or null
  // structure
  const NodeDev* nodes;
  const ProbDev* probs;
  const SubDev* subs;
  const MacroDev* macros;
  const int* border;
  const int* children;
  const int* rel;
  const int* dtype;
  const int* dsrc;
  const int* bgrp;           // per position: deluxe entity of a root-border DOF, -1 otherwise
  const int* elpos;
  const int* elptr;
  const int* pos_of_vdof;
  const int* sub_elems;
  const int64_t* vdof;
  const int* vadj_ptr;
  const int* vadj;
  const int* vcon_ptr;
  const int* vcon_id;
  const double* vcon_coef;
  const int64_t* press;
  const double* wmean;
  const int* iface;
  const int64_t* coarse;
  const int* elloc;          // per subdomain element column -> local index (vdof or nv + pressure)
  const int* elloc_ptr;      // per subdomain: local element -> offset into its elloc table
  // macro entity data
  const int64_t* mdofs;
  const double* hv;
  const double* tau;
  const int* share;
  const int* gpos;           // (entity, sharing subdomain) -> Neumann positions of its DOFs
  const int* gif;            // (entity, sharing subdomain) -> local interface index of its DOFs
  const double* deluxe;      // D^(share[0]) per deluxe face
  const double* deluxe_e;    // D^(s) for every sharing subdomain s per deluxe edge
  int64_t ncv, nc;           // coarse velocity coordinates, all coarse coordinates
};

}  // namespace vb

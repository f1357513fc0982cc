// Per-element VEM construction (Sec. 3): face projectors Pi^nabla_{k,f},
// Pi^0_{k+1,f} (Eq. faceSpace), element divergence, Pi^nabla_{k,K},
// Pi^0_{k-1} grad, Pi^0_k (Eq. velSpace), the local stiffness
// a_h^K = consistency + stabilization (Eq. discreteA) and B_K.
//
// One cooperating group of `nt` threads (a CTA) builds one element, written
// against a tiny execution interface (thread id, count, barrier).
//
// Polynomial facts used (all in scaled monomials xi = (x - x_K)/h_K):
//  * any homogeneous w in [P_d]^3 splits as
//      w = grad( (xi.w)/(d+1) ) - xi ^ (curl w)/(d+1),
//    which gives the moments int v.w from divergence/boundary data and from
//    moments against xi ^ [P_{d-1}]^3 (D4 for d-1 <= k-3, enhancement of
//    Eq. velSpace for d-1 in {k-2, k-1});
//  * int_K v.grad q = -int_K div v q + int_dK (v.n) q, and boundary traces are
//    replaced by Pi^0_{k+1,f} v on each face (exact against P_{k+1}(f)).
#pragma once
#include <cmath>
#include "common.h"
#include "system.h"
#include "launch.h"

namespace vb {

using Exec = KExec;

// element-independent tables (quadrature rules, monomial exponents)
struct ElemTables {
  Exp3 e3[kMaxMono3];
  Exp2 e2[kMaxMono2];
  double gl[4];            // interior Gauss-Lobatto nodes (k-1 used)
  int nq_edge;
  double qe_x[8], qe_w[8];     // edge rule on [0,1]
  int nq_face;
  double qf_x[8], qf_w[8];     // 1D Gauss nodes for the collapsed triangle rule
  int nq_vol;
  double qv_x[8], qv_w[8];     // 1D Gauss nodes for the collapsed tetrahedron rule
};

template <int K>
struct ElemSizes {
  static constexpr int NP0 = pdim3(K - 1);     // pressure / divergence space
  static constexpr int NP1 = pdim3(K);
  static constexpr int NP2 = pdim3(K + 1);
  static constexpr int NMOM = pdim3(2 * K);    // volume moments needed
  static constexpr int NF1 = pdim2(K);
  static constexpr int NF2 = pdim2(K + 1);
  static constexpr int NFM = pdim2(K - 2);
  static constexpr int NFMOM = pdim2(2 * K + 2);
  static constexpr int NL = pdim3(K - 2);
  static constexpr int NQ3 = pdim3(K - 3);
  static constexpr int N4 = n_d4(K);
  static constexpr int N5 = n_d5(K);
  static constexpr int NSMAX = kMaxFaceVerts * K + NFM;   // face-local DOFs per component
  // quadrature: collapsed Gauss rules with NQF (triangle) and NQV
  // (tetrahedron) points per direction (exact to degree 2k+2 and 2k)
  static constexpr int NQF = (2 * K + 5) / 2;
  static constexpr int NQV = K + 2;
  // tetrahedra of the volume rule tabulated at once
  static constexpr int TCH = 16;
  // point tables: volume (TCH tets: weight and 3 coordinates; partial
  // moments per tet slot) and face (one fan triangle: weight, 5 coordinates,
  // the 3D monomials of P_{k+1} and the face monomials of degree <= 2k+2)
  static constexpr int TABV = TCH * NQV * NQV * NQV * 4 + NMOM * TCH;
  static constexpr int TABF = NQF * NQF * (6 + NP2 + NFMOM);
  static constexpr int TAB = TABV > TABF ? TABV : TABF;
};

// shared (fast) working set of one element
template <int K>
struct ElemShared {
  using S = ElemSizes<K>;
  double X[kMaxElemVerts][3];
  double xK[3], hK, vol;
  double fn[kMaxElemFaces][3], ft1[kMaxElemFaces][3], ft2[kMaxElemFaces][3], fxc[kMaxElemFaces][3];
  double fh[kMaxElemFaces], farea[kMaxElemFaces], ifarea[kMaxElemFaces];
  // face-local coordinates (s, t) = fw (xi1, xi2), xi = ((x - xc).t1, (x - xc).t2):
  // fw = Sigma^{-1/2} / sqrt(24), Sigma the second moments of the face about xc
  double fw[kMaxElemFaces][4];
  double mu[S::NMOM];
  double Minv0[S::NP0 * S::NP0];   // inverse mass on P_{k-1}
  double Minv1[S::NP1 * S::NP1];   // inverse mass on P_k
  double Ginv[S::NP1 * S::NP1];    // inverse of the Pi^nabla_k system
  double bndm[S::NP1];             // int_dK m_g
  double big[S::NP1 * S::NP1];     // temporary for the inversions
  // per-face work
  double nu2[S::NFMOM];
  double G2[S::NF1 * S::NF1];
  double MF[S::NF2 * S::NF2];
  double W[S::NP2 * S::NF2];
  double PiN[S::NF1 * S::NSMAX];
  double Pi0[S::NF2 * S::NSMAX];
  double rhs[S::NF2 * S::NSMAX];
  double red[256];
};

// global scratch layout of one element (sizes in doubles)
template <int K>
struct ElemScratch {
  using S = ElemSizes<K>;
  static VB_HD size_t face_block() { return (size_t)S::NP2 * S::NSMAX; }
  static VB_HD size_t size(int nK) {
    return kMaxElemFaces * face_block() + (size_t)nK *
               (S::NP0 + S::NP2 + 3 * S::NL + 3 * S::NP1 + 12 * S::NP0 + 3 * S::NP1 + 3 * S::NP1) +
           2 * (size_t)nK * nK + S::TAB + (size_t)kMaxElemFaces * S::NP1 * S::NFM;
  }
};

VB_HD inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// 1/n for the small positive integers of the monomial calculus (folded
// constants instead of FP64 divisions)
VB_HD inline double inv_small(int n) {
  switch (n) {
    case 1: return 1.0;
    case 2: return 1.0 / 2;
    case 3: return 1.0 / 3;
    case 4: return 1.0 / 4;
    case 5: return 1.0 / 5;
    case 6: return 1.0 / 6;
    case 7: return 1.0 / 7;
    case 8: return 1.0 / 8;
    case 9: return 1.0 / 9;
    case 10: return 1.0 / 10;
    case 11: return 1.0 / 11;
    case 12: return 1.0 / 12;
    case 13: return 1.0 / 13;
    default: return 1.0 / n;
  }
}

VB_HD inline double ipow(double x, int p) {
  double r = 1.0;
  for (int i = 0; i < p; ++i) r *= x;
  return r;
}

// In-place Gauss-Jordan inverse with partial pivoting of an n x n row-major
// matrix (one thread).  Returns false on a zero pivot.
VB_HD inline bool small_inverse(double* M, double* Inv, int n) {
  for (int i = 0; i < n * n; ++i) Inv[i] = 0.0;
  for (int i = 0; i < n; ++i) Inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = M[c * n + c] < 0 ? -M[c * n + c] : M[c * n + c];
    for (int r = c + 1; r < n; ++r) {
      double v = M[r * n + c] < 0 ? -M[r * n + c] : M[r * n + c];
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        double t = M[c * n + j]; M[c * n + j] = M[p * n + j]; M[p * n + j] = t;
        t = Inv[c * n + j]; Inv[c * n + j] = Inv[p * n + j]; Inv[p * n + j] = t;
      }
    double d = 1.0 / M[c * n + c];
    for (int j = 0; j < n; ++j) { M[c * n + j] *= d; Inv[c * n + j] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { M[r * n + j] -= f * M[c * n + j]; Inv[r * n + j] -= f * Inv[c * n + j]; }
    }
  }
  return true;
}

// The same Gauss-Jordan inversion run by one warp (lanes 0..31 call it;
// every lane scans for the pivot, each lane eliminates whole rows): the
// operations on every entry, and their order, are those of small_inverse.
VB_HD inline bool small_inverse_warp(double* M, double* Inv, int n, int lane) {
#ifdef __CUDA_ARCH__
  for (int i = lane; i < n * n; i += 32) Inv[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncwarp();
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = M[c * n + c] < 0 ? -M[c * n + c] : M[c * n + c];
    for (int r = c + 1; r < n; ++r) {
      double v = M[r * n + c] < 0 ? -M[r * n + c] : M[r * n + c];
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return false;
    __syncwarp();
    if (p != c)
      for (int j = lane; j < n; j += 32) {
        double t = M[c * n + j]; M[c * n + j] = M[p * n + j]; M[p * n + j] = t;
        t = Inv[c * n + j]; Inv[c * n + j] = Inv[p * n + j]; Inv[p * n + j] = t;
      }
    __syncwarp();
    const double d = 1.0 / M[c * n + c];
    __syncwarp();
    for (int j = lane; j < n; j += 32) { M[c * n + j] *= d; Inv[c * n + j] *= d; }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { M[r * n + j] -= f * M[c * n + j]; Inv[r * n + j] -= f * Inv[c * n + j]; }
    }
    __syncwarp();
  }
  return true;
#else
  (void)lane;
  return small_inverse(M, Inv, n);
#endif
}

template <int K>
struct ElemBuilder {
  using S = ElemSizes<K>;
  const ElemRec& R;
  const double* xyz;
  const ElemTables& T;
  ElemShared<K>& sh;
  double* scr;
  int nK;
  int off_e, off_f, off_4, off_5;
  Exec ex;
  // scratch views
  double *Y, *DIV, *GM, *VML, *PiN, *Rs, *E, *VMH, *Dm, *Pm, *Tb, *FM;

  VB_HD ElemBuilder(const ElemRec& r, const double* x, const ElemTables& t, ElemShared<K>& s, double* sc, Exec e)
      : R(r), xyz(x), T(t), sh(s), scr(sc), ex(e) {
    nK = R.nK;
    off_e = 3 * R.nv;
    off_f = off_e + R.ne * 3 * (K - 1);
    off_4 = off_f + R.nf * 3 * S::NFM;
    off_5 = off_4 + S::N4;
    size_t o = 0;
    Y = scr + o;   o += kMaxElemFaces * ElemScratch<K>::face_block();
    DIV = scr + o; o += (size_t)S::NP0 * nK;
    GM = scr + o;  o += (size_t)S::NP2 * nK;
    VML = scr + o; o += (size_t)3 * S::NL * nK;
    PiN = scr + o; o += (size_t)3 * S::NP1 * nK;
    Rs = scr + o;  o += (size_t)6 * S::NP0 * nK;
    E = scr + o;   o += (size_t)6 * S::NP0 * nK;
    VMH = scr + o; o += (size_t)3 * S::NP1 * nK;
    Dm = scr + o;  o += (size_t)3 * S::NP1 * nK;
    Pm = scr + o;  o += (size_t)2 * nK * nK;
    Tb = scr + o;  o += S::TAB;
    FM = scr + o;  o += (size_t)kMaxElemFaces * S::NP1 * S::NFM;
  }

  VB_HD double mu(int a, int b, int c) const { return sh.mu[idx3(a, b, c)]; }
  // int_K m_p m_q
  VB_HD double mass(int p, int q) const {
    const Exp3 &A = T.e3[p], &B = T.e3[q];
    return mu(A.a + B.a, A.b + B.b, A.c + B.c);
  }
  VB_HD int ns(int f) const { return R.fnv[f] * K + S::NFM; }

  // ---------------------------------------------------------------- geometry
  VB_HD void geometry() {
    if (ex.tid == 0) {
      double c[3] = {0, 0, 0};
      for (int i = 0; i < R.nv; ++i)
        for (int d = 0; d < 3; ++d) {
          sh.X[i][d] = xyz[3 * R.vert[i] + d];
          c[d] += sh.X[i][d];
        }
      for (int d = 0; d < 3; ++d) sh.xK[d] = c[d] / R.nv;
      double h2 = 0;
      for (int i = 0; i < R.nv; ++i)
        for (int j = i + 1; j < R.nv; ++j) {
          double s = 0;
          for (int d = 0; d < 3; ++d) s += (sh.X[i][d] - sh.X[j][d]) * (sh.X[i][d] - sh.X[j][d]);
          h2 = s > h2 ? s : h2;
        }
      sh.hK = sqrt(h2);
    }
    ex.sync();
    // faces independently, one thread each
    for (int f = ex.tid; f < R.nf; f += ex.nt) {
      {
        int m = R.fnv[f];
        double nrm[3] = {0, 0, 0}, xc[3] = {0, 0, 0}, h2f = 0;
        for (int i = 0; i < m; ++i) {
          const double* a = sh.X[R.floopv[f][i]];
          const double* b = sh.X[R.floopv[f][(i + 1) % m]];
          double cr[3];
          cross3(a, b, cr);
          for (int d = 0; d < 3; ++d) { nrm[d] += cr[d]; xc[d] += a[d]; }
          for (int j = i + 1; j < m; ++j) {
            const double* bb = sh.X[R.floopv[f][j]];
            double s = 0;
            for (int d = 0; d < 3; ++d) s += (a[d] - bb[d]) * (a[d] - bb[d]);
            h2f = s > h2f ? s : h2f;
          }
        }
        double ln = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        sh.farea[f] = 0.5 * ln;
        sh.fh[f] = sqrt(h2f);
        const double* p0 = sh.X[R.floopv[f][0]];
        const double* p1 = sh.X[R.floopv[f][1]];
        double t1[3], dd = 0;
        for (int d = 0; d < 3; ++d) { sh.fn[f][d] = nrm[d] / ln; t1[d] = p1[d] - p0[d]; }
        for (int d = 0; d < 3; ++d) dd += t1[d] * sh.fn[f][d];
        double lt = 0;
        for (int d = 0; d < 3; ++d) { t1[d] -= dd * sh.fn[f][d]; lt += t1[d] * t1[d]; }
        lt = sqrt(lt);
        for (int d = 0; d < 3; ++d) { sh.ft1[f][d] = t1[d] / lt; sh.fxc[f][d] = xc[d] / m; }
        cross3(sh.fn[f], sh.ft1[f], sh.ft2[f]);
        face_whitening(f);
      }
    }
    ex.sync();
  }

  // Second moments Sigma = (1/|f|) int_f xi xi^T of the face about xc in the
  // (t1, t2) frame, exact on the fan triangles from loop vertex 0, and
  // fw = Sigma^{-1/2} / sqrt(24) in closed form: sqrt(S) = (S + d I) / tau
  // with d = sqrt(det S), tau = sqrt(tr S + 2 d).  Polynomial spaces on the
  // face are invariant under this linear map of the centred coordinates; the
  // scaled monomials stay well conditioned on thin faces.
  VB_HD void face_whitening(int f) {
    const int m = R.fnv[f];
    const double* xc = sh.fxc[f];
    const double *t1 = sh.ft1[f], *t2 = sh.ft2[f];
    double q[kMaxFaceVerts][2];
    for (int i = 0; i < m; ++i) {
      const double* P = sh.X[R.floopv[f][i]];
      double dx[3] = {P[0] - xc[0], P[1] - xc[1], P[2] - xc[2]};
      q[i][0] = dx[0] * t1[0] + dx[1] * t1[1] + dx[2] * t1[2];
      q[i][1] = dx[0] * t2[0] + dx[1] * t2[1] + dx[2] * t2[2];
    }
    double s00 = 0, s01 = 0, s11 = 0, area = 0;
    for (int i = 1; i < m - 1; ++i) {
      const double *a = q[0], *b = q[i], *c = q[i + 1];
      double ar = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));
      double sm0 = a[0] + b[0] + c[0], sm1 = a[1] + b[1] + c[1];
      double w = ar / 12.0;
      s00 += w * (a[0] * a[0] + b[0] * b[0] + c[0] * c[0] + sm0 * sm0);
      s01 += w * (a[0] * a[1] + b[0] * b[1] + c[0] * c[1] + sm0 * sm1);
      s11 += w * (a[1] * a[1] + b[1] * b[1] + c[1] * c[1] + sm1 * sm1);
      area += ar;
    }
    s00 /= area;
    s01 /= area;
    s11 /= area;
    double d = sqrt(s00 * s11 - s01 * s01);
    double tau = sqrt(s00 + s11 + 2.0 * d);
    double sc = 1.0 / (d * tau * sqrt(24.0));
    sh.fw[f][0] = (s11 + d) * sc;
    sh.fw[f][1] = -s01 * sc;
    sh.fw[f][2] = -s01 * sc;
    sh.fw[f][3] = (s00 + d) * sc;
  }

  // face-local coordinates of the point x on face f
  VB_HD void face_st(int f, const double* x, double& s, double& t) const {
    const double* xc = sh.fxc[f];
    const double *t1 = sh.ft1[f], *t2 = sh.ft2[f];
    double dx[3] = {x[0] - xc[0], x[1] - xc[1], x[2] - xc[2]};
    double a = dx[0] * t1[0] + dx[1] * t1[1] + dx[2] * t1[2];
    double b = dx[0] * t2[0] + dx[1] * t2[1] + dx[2] * t2[2];
    s = sh.fw[f][0] * a + sh.fw[f][1] * b;
    t = sh.fw[f][2] * a + sh.fw[f][3] * b;
  }

  // ------------------------------------------------ volume moments mu_a = int xi^a
  // Tetrahedra (x_K, A, B, C) of the fan of every face (outward loop); the
  // points of up to TCH tetrahedra are tabulated (weight, scaled coordinates),
  // then every (moment, tetrahedron) pair sums over its points, and each
  // moment adds its tetrahedra in order.
  VB_HD void tet_of(int tet, int& f, int& t) const {
    f = 0;
    while (tet >= R.fnv[f] - 2) { tet -= R.fnv[f] - 2; ++f; }
    t = 1 + tet;
  }
  VB_HD void volume_moments() {
    constexpr int NQ = S::NQV, NPT = NQ * NQ * NQ, CH = S::TCH;
    double* VT = Tb;                   // [CH][NPT][4]
    double* PART = Tb + CH * NPT * 4;  // [NMOM][CH]
    const double hinv = 1.0 / sh.hK;
    int ntet = 0;
    for (int f = 0; f < R.nf; ++f) ntet += R.fnv[f] - 2;
    for (int i = ex.tid; i < S::NMOM * CH; i += ex.nt) PART[i] = 0.0;
    for (int c0 = 0; c0 < ntet; c0 += CH) {
      ex.sync();
      for (int item = ex.tid; item < CH * NPT; item += ex.nt) {
        const int j = item / NPT, q = item % NPT;
        if (c0 + j >= ntet) continue;
        int f, t;
        tet_of(c0 + j, f, t);
        const int m = R.fnv[f];
        int i0 = 0, i1 = t, i2 = t + 1;
        if (R.fsign[f] < 0) { i0 = m - 1; i1 = m - 1 - t; i2 = m - 2 - t; }
        const double* A = sh.X[R.floopv[f][i0]];
        const double* B = sh.X[R.floopv[f][i1]];
        const double* C = sh.X[R.floopv[f][i2]];
        double a1[3], b1[3], c1[3];
        for (int d = 0; d < 3; ++d) { a1[d] = A[d] - sh.xK[d]; b1[d] = B[d] - sh.xK[d]; c1[d] = C[d] - sh.xK[d]; }
        double cr[3];
        cross3(b1, c1, cr);
        const double det = a1[0] * cr[0] + a1[1] * cr[1] + a1[2] * cr[2];
        const int iu = q / (NQ * NQ), iv = (q / NQ) % NQ, iw = q % NQ;
        const double U = T.qv_x[iu], V = T.qv_x[iv], Wd = T.qv_x[iw];
        const double x = U, y = V * (1 - U), z = Wd * (1 - U) * (1 - V);
        double* o = VT + (size_t)item * 4;
        o[0] = T.qv_w[iu] * T.qv_w[iv] * T.qv_w[iw] * (1 - U) * (1 - U) * (1 - V) * det;
        for (int d = 0; d < 3; ++d) o[1 + d] = (x * a1[d] + y * b1[d] + z * c1[d]) * hinv;
      }
      ex.sync();
      for (int item = ex.tid; item < S::NMOM * CH; item += ex.nt) {
        const int a = item / CH, j = item % CH;
        if (c0 + j >= ntet) continue;
        const Exp3 ea = T.e3[a];
        const double* v = VT + (size_t)j * NPT * 4;
        double acc = 0.0;
        for (int q = 0; q < NPT; ++q, v += 4) acc += v[0] * ipow(v[1], ea.a) * ipow(v[2], ea.b) * ipow(v[3], ea.c);
        PART[item] += acc;
      }
    }
    ex.sync();
    for (int a = ex.tid; a < S::NMOM; a += ex.nt) {
      double acc = 0.0;
      for (int j = 0; j < CH; ++j) acc += PART[a * CH + j];
      sh.mu[a] = acc;
    }
    ex.sync();
    if (ex.tid == 0) sh.vol = sh.mu[0];
    ex.sync();
  }

  // inverse mass matrices and the Pi^nabla_k system
  VB_HD bool volume_systems() {
    double* tmp = sh.big;
    bool ok = true;
    for (int idx = ex.tid; idx < S::NP0 * S::NP0; idx += ex.nt) tmp[idx] = mass(idx / S::NP0, idx % S::NP0);
    ex.sync();
    if (ex.tid < 32) ok = small_inverse_warp(tmp, sh.Minv0, S::NP0, ex.tid);
    ex.sync();
    for (int idx = ex.tid; idx < S::NP1 * S::NP1; idx += ex.nt) tmp[idx] = mass(idx / S::NP1, idx % S::NP1);
    ex.sync();
    if (ex.tid < 32) ok = small_inverse_warp(tmp, sh.Minv1, S::NP1, ex.tid) && ok;
    ex.sync();
    return ok;
  }

  // ------------------------------------------------ faces
  VB_HD bool face(int f) {
    const int m = R.fnv[f];
    const int nsf = ns(f);
    const double *t1 = sh.ft1[f], *t2 = sh.ft2[f];
    const double* fw = sh.fw[f];
    // metric of the face-local coordinates: grad_x m . grad_x n = grad_st m^T (fw fw^T) grad_st n
    const double g00 = fw[0] * fw[0] + fw[1] * fw[1];
    const double g01 = fw[0] * fw[2] + fw[1] * fw[3];
    const double g11 = fw[2] * fw[2] + fw[3] * fw[3];
    // face quadrature (fan from loop vertex 0, collapsed Gauss); 2D moments
    // nu_g = int_f s^g1 t^g2 and W[a][b] = int_f m3_a m2_b.  Per fan
    // triangle the points are tabulated (weight, (s, t), scaled xi), then the
    // monomials at every point, then each moment sums over the points.
    {
      constexpr int NQ = S::NQF, NPT = NQ * NQ, NMT = S::NP2 + S::NFMOM;
      double* FT = Tb;                  // [NPT][6]: w, s, t, xi
      double* M3 = Tb + NPT * 6;        // [NPT][NP2]
      double* M2 = M3 + NPT * S::NP2;   // [NPT][NFMOM]
      const double hk = 1.0 / sh.hK;
      for (int idx = ex.tid; idx < S::NFMOM + S::NP2 * S::NF2; idx += ex.nt) {
        if (idx < S::NFMOM) sh.nu2[idx] = 0.0;
        else sh.W[idx - S::NFMOM] = 0.0;
      }
      const double* P0 = sh.X[R.floopv[f][0]];
      for (int t = 1; t < m - 1; ++t) {
        const double* P1 = sh.X[R.floopv[f][t]];
        const double* P2 = sh.X[R.floopv[f][t + 1]];
        ex.sync();
        for (int q = ex.tid; q < NPT; q += ex.nt) {
          double u1[3], u2[3], cr[3];
          for (int d = 0; d < 3; ++d) { u1[d] = P1[d] - P0[d]; u2[d] = P2[d] - P0[d]; }
          cross3(u1, u2, cr);
          const double J = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
          const int iu = q / NQ, iv = q % NQ;
          const double U = T.qf_x[iu], V = T.qf_x[iv] * (1 - U);
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = P0[d] + U * u1[d] + V * u2[d];
          double* o = FT + q * 6;
          o[0] = T.qf_w[iu] * T.qf_w[iv] * (1 - U) * J;
          face_st(f, x, o[1], o[2]);
          for (int d = 0; d < 3; ++d) o[3 + d] = (x[d] - sh.xK[d]) * hk;
        }
        ex.sync();
        for (int item = ex.tid; item < NPT * NMT; item += ex.nt) {
          const int q = item / NMT, jm = item % NMT;
          const double* o = FT + q * 6;
          if (jm < S::NP2) {
            const Exp3 ea = T.e3[jm];
            M3[q * S::NP2 + jm] = ipow(o[3], ea.a) * ipow(o[4], ea.b) * ipow(o[5], ea.c);
          } else {
            const Exp2 eb = T.e2[jm - S::NP2];
            M2[q * S::NFMOM + jm - S::NP2] = ipow(o[1], eb.a) * ipow(o[2], eb.b);
          }
        }
        ex.sync();
        for (int idx = ex.tid; idx < S::NFMOM + S::NP2 * S::NF2; idx += ex.nt) {
          double acc = 0.0;
          if (idx < S::NFMOM) {
            for (int q = 0; q < NPT; ++q) acc += FT[q * 6] * M2[q * S::NFMOM + idx];
            sh.nu2[idx] += acc;
          } else {
            const int a = (idx - S::NFMOM) / S::NF2, b = (idx - S::NFMOM) % S::NF2;
            for (int q = 0; q < NPT; ++q) acc += FT[q * 6] * M3[q * S::NP2 + a] * M2[q * S::NFMOM + b];
            sh.W[a * S::NF2 + b] += acc;
          }
        }
      }
    }
    ex.sync();
    // int_f m3_a m2_b for a in P_k, b in P_{k-2}(f), kept for the DOFs of the
    // [P_k]^3 basis
    for (int idx = ex.tid; idx < S::NP1 * S::NFM; idx += ex.nt)
      FM[(size_t)f * S::NP1 * S::NFM + idx] = sh.W[(idx / S::NFM) * S::NF2 + idx % S::NFM];
    // Pi^nabla_{k,f}: G2 c = rhs, rows b >= 1: int grad m_b . grad m_g;
    // row 0: int_df m_g.  rhs: -int Lap m_b v + sum_e int_e d_n m_b v; row 0 int_df v
    for (int idx = ex.tid; idx < S::NF1 * S::NF1; idx += ex.nt) {
      int b = idx / S::NF1, g = idx % S::NF1;
      const Exp2 eb = T.e2[b], eg = T.e2[g];
      double v = 0.0;
      if (b > 0) {
        if (eb.a > 0 && eg.a > 0) v += g00 * eb.a * eg.a * sh.nu2[idx2(eb.a + eg.a - 2, eb.b + eg.b)];
        if (eb.b > 0 && eg.b > 0) v += g11 * eb.b * eg.b * sh.nu2[idx2(eb.a + eg.a, eb.b + eg.b - 2)];
        const int mx = eb.a * eg.b + eb.b * eg.a;   // d_s m_b d_t m_g + d_t m_b d_s m_g
        if (mx > 0) v += g01 * mx * sh.nu2[idx2(eb.a + eg.a - 1, eb.b + eg.b - 1)];
      }
      sh.G2[idx] = v;
    }
    for (int idx = ex.tid; idx < S::NF1 * nsf; idx += ex.nt) sh.rhs[idx] = 0.0;
    ex.sync();
    // one thread per basis function b of P_k(f): it fills row b of the
    // right-hand side and entry b of row 0 of G2, in the same order as a
    // single thread would (Laplacian terms, then edge by edge, point by point)
    for (int b = ex.tid; b < S::NF1; b += ex.nt) {
      const Exp2 eb = T.e2[b];
      // interior moments: -int_f Lap m_b v = -|f| sum_g L[g][b] s_g
      if (b > 0) {
        if (eb.a >= 2) sh.rhs[b * nsf + m * K + idx2(eb.a - 2, eb.b)] -= sh.farea[f] * g00 * eb.a * (eb.a - 1);
        if (eb.a >= 1 && eb.b >= 1)
          sh.rhs[b * nsf + m * K + idx2(eb.a - 1, eb.b - 1)] -= sh.farea[f] * 2.0 * g01 * eb.a * eb.b;
        if (eb.b >= 2) sh.rhs[b * nsf + m * K + idx2(eb.a, eb.b - 2)] -= sh.farea[f] * g11 * eb.b * (eb.b - 1);
      }
      double g2b = 0.0;
      // edges: Gauss points, Lagrange basis on (0, interior GL nodes, 1)
      double nodes[K + 1];
      nodes[0] = 0.0;
      for (int j = 0; j < K - 1; ++j) nodes[1 + j] = T.gl[j];
      nodes[K] = 1.0;
      for (int i = 0; i < m; ++i) {
        const double* A = sh.X[R.floopv[f][i]];
        const double* B = sh.X[R.floopv[f][(i + 1) % m]];
        double dvec[3], le = 0;
        for (int d = 0; d < 3; ++d) { dvec[d] = B[d] - A[d]; le += dvec[d] * dvec[d]; }
        le = sqrt(le);
        double du[3] = {dvec[0] / le, dvec[1] / le, dvec[2] / le};
        double ne[3];
        cross3(du, sh.fn[f], ne);
        // d_n m = (fw (ne.t1, ne.t2)) . grad_st m
        double e1 = ne[0] * t1[0] + ne[1] * t1[1] + ne[2] * t1[2];
        double e2 = ne[0] * t2[0] + ne[1] * t2[1] + ne[2] * t2[2];
        double n1 = fw[0] * e1 + fw[1] * e2;
        double n2 = fw[2] * e1 + fw[3] * e2;
        int sidx[K + 1];
        sidx[0] = i;
        for (int j = 0; j < K - 1; ++j) sidx[1 + j] = m + i * (K - 1) + j;
        sidx[K] = (i + 1) % m;
        for (int q = 0; q < T.nq_edge; ++q) {
          double tq = T.qe_x[q], wq = T.qe_w[q] * le;
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = A[d] + tq * dvec[d];
          double s, tt;
          face_st(f, x, s, tt);
          double lag[K + 1];
          for (int aa = 0; aa <= K; ++aa) {
            double l = 1.0;
            for (int bb = 0; bb <= K; ++bb)
              if (bb != aa) l *= (tq - nodes[bb]) / (nodes[aa] - nodes[bb]);
            lag[aa] = l;
          }
          double mb = ipow(s, eb.a) * ipow(tt, eb.b);
          if (b == 0) {
            for (int aa = 0; aa <= K; ++aa) sh.rhs[sidx[aa]] += wq * lag[aa];
          } else {
            double ds = eb.a > 0 ? eb.a * ipow(s, eb.a - 1) * ipow(tt, eb.b) : 0.0;
            double dt = eb.b > 0 ? eb.b * ipow(s, eb.a) * ipow(tt, eb.b - 1) : 0.0;
            double dn = ds * n1 + dt * n2;
            for (int aa = 0; aa <= K; ++aa) sh.rhs[b * nsf + sidx[aa]] += wq * dn * lag[aa];
          }
          g2b += wq * mb;     // row 0 of G2: int_df m_b
        }
      }
      sh.G2[b] = g2b;
    }
    ex.sync();
    // solve (one thread inverts; all apply)
    double* G2inv = sh.MF;   // borrowed until the face mass is formed
    bool ok = true;
    if (ex.tid < 32) ok = small_inverse_warp(sh.G2, G2inv, S::NF1, ex.tid);
    ex.sync();
    for (int idx = ex.tid; idx < S::NF1 * nsf; idx += ex.nt) {
      int b = idx / nsf, s = idx % nsf;
      double acc = 0.0;
      for (int g = 0; g < S::NF1; ++g) acc += G2inv[b * S::NF1 + g] * sh.rhs[g * nsf + s];
      sh.PiN[idx] = acc;
    }
    ex.sync();
    // Pi^0_{k+1,f}: face mass; rhs rows < NFM from the moments, others from Pi^nabla
    double* MFm = sh.rhs;    // rhs consumed: reuse for the face mass
    for (int idx = ex.tid; idx < S::NF2 * S::NF2; idx += ex.nt) {
      int b = idx / S::NF2, g = idx % S::NF2;
      MFm[idx] = sh.nu2[idx2(T.e2[b].a + T.e2[g].a, T.e2[b].b + T.e2[g].b)];
    }
    ex.sync();
    if (ex.tid < 32) ok = small_inverse_warp(MFm, sh.MF, S::NF2, ex.tid) && ok;
    ex.sync();
    // rhs for Pi^0 into Pi0 (temporarily), then multiply by MF^{-1} into rhs
    for (int idx = ex.tid; idx < S::NF2 * nsf; idx += ex.nt) {
      int b = idx / nsf, s = idx % nsf;
      double v = 0.0;
      if (b < S::NFM) {
        v = (s == m * K + b) ? sh.farea[f] : 0.0;
      } else {
        for (int g = 0; g < S::NF1; ++g)
          v += sh.nu2[idx2(T.e2[b].a + T.e2[g].a, T.e2[b].b + T.e2[g].b)] * sh.PiN[g * nsf + s];
      }
      sh.Pi0[idx] = v;
    }
    ex.sync();
    for (int idx = ex.tid; idx < S::NF2 * nsf; idx += ex.nt) {
      int b = idx / nsf, s = idx % nsf;
      double acc = 0.0;
      for (int g = 0; g < S::NF2; ++g) acc += sh.MF[b * S::NF2 + g] * sh.Pi0[g * nsf + s];
      sh.rhs[idx] = acc;
    }
    ex.sync();
    // Y_f = W Pi0_f : int_f m3_a (Pi^0_{k+1,f} v)  for a in P_{k+1}
    double* Yf = Y + (size_t)f * ElemScratch<K>::face_block();
    for (int idx = ex.tid; idx < S::NP2 * nsf; idx += ex.nt) {
      int a = idx / nsf, s = idx % nsf;
      double acc = 0.0;
      for (int b = 0; b < S::NF2; ++b) acc += sh.W[a * S::NF2 + b] * sh.rhs[b * nsf + s];
      Yf[idx] = acc;
    }
    // int_f m3_g for g in P_k (row 0 of the Pi^nabla_K system)
    if (ex.tid == 0) {
      for (int g = 0; g < S::NP1; ++g) sh.bndm[g] += sh.W[g * S::NF2 + 0];
    }
    ex.sync();
    return ok;
  }

  // boundary functional entry: column `col` of  int_dK v_c m_a (n_j)  (j < 0: no normal)
  VB_HD double bnd(int col, int c, int a, int j) const {
    double acc = 0.0;
    // decode the entity of col
    if (col < off_e) {
      int lv = col / 3, cc = col % 3;
      if (cc != c) return 0.0;
      for (int f = 0; f < R.nf; ++f) {
        int m = R.fnv[f];
        for (int i = 0; i < m; ++i)
          if (R.floopv[f][i] == lv) {
            double cf = j < 0 ? 1.0 : R.fsign[f] * sh.fn[f][j];
            acc += cf * Y[(size_t)f * ElemScratch<K>::face_block() + a * ns(f) + i];
          }
      }
      return acc;
    }
    if (col < off_f) {
      int r = col - off_e;
      int le = r / (3 * (K - 1));
      int jj = (r / 3) % (K - 1), cc = r % 3;
      if (cc != c) return 0.0;
      for (int f = 0; f < R.nf; ++f) {
        int m = R.fnv[f];
        for (int i = 0; i < m; ++i)
          if (R.floope[f][i] == le) {
            int jt = R.floopdir[f][i] ? jj : (K - 2 - jj);
            double cf = j < 0 ? 1.0 : R.fsign[f] * sh.fn[f][j];
            acc += cf * Y[(size_t)f * ElemScratch<K>::face_block() + a * ns(f) + m + i * (K - 1) + jt];
          }
      }
      return acc;
    }
    if (col < off_4) {
      int r = col - off_f;
      int f = r / (3 * S::NFM);
      int b = (r / 3) % S::NFM, t = r % 3;
      double wv = t == 0 ? sh.fn[f][c] : (t == 1 ? sh.ft1[f][c] : sh.ft2[f][c]);
      double cf = j < 0 ? 1.0 : R.fsign[f] * sh.fn[f][j];
      return cf * wv * Y[(size_t)f * ElemScratch<K>::face_block() + a * ns(f) + R.fnv[f] * K + b];
    }
    return 0.0;
  }

  // D4 functional: column pattern of  int_K v . (xi ^ (m_b e_i)), b in P_{k-3}
  // (dependent generator (xi_3, z) at k = 4 replaced by minus the other two)
  VB_HD double d4(int col, int b, int i) const {
    if (col < off_4 || col >= off_5) return 0.0;
    int jcol = col - off_4;
    int g = b * 3 + i;
    if (K == 4 && g == 3 * 3 + 2) {
      // -(g(xi_1, x) + g(xi_2, y)) : generators 3*1+0 and 3*2+1
      double v = 0.0;
      if (jcol == 3) v -= 1.0;
      if (jcol == 7) v -= 1.0;
      return v * sh.vol;
    }
    return (jcol == g) ? sh.vol : 0.0;
  }

  // moment of v against xi ^ (m_b e_i) for deg(b) >= k-2 via Pi^nabla (enhancement)
  VB_HD double enh(int col, int b, int i) const {
    // (xi ^ e_i m_b)_comp = eps(comp, j, i) xi_j m_b
    double acc = 0.0;
    for (int comp = 0; comp < 3; ++comp)
      for (int jd = 0; jd < 3; ++jd) {
        int eps = 0;
        if (comp == jd || jd == i || comp == i) continue;
        eps = ((comp + 1) % 3 == jd) ? 1 : -1;   // cyclic (comp, jd, i)
        const Exp3 eb = T.e3[b];
        for (int g = 0; g < S::NP1; ++g) {
          const Exp3 eg = T.e3[g];
          int ea = eg.a + eb.a + (jd == 0), ebb = eg.b + eb.b + (jd == 1), ec = eg.c + eb.c + (jd == 2);
          acc += eps * PiN[((size_t)comp * S::NP1 + g) * nK + col] * mu(ea, ebb, ec);
        }
      }
    return acc;
  }

  // int_K v . (m_b e_c) for the vector monomial of degree d = |b|, column col
  VB_HD double vecmom(int col, int c, int b, bool use_enh) const {
    const Exp3 eb = T.e3[b];
    int d = eb.a + eb.b + eb.c;
    double hK = sh.hK;
    // gradient part: Q = xi_c m_b / (d+1);  int v . grad_xi Q = h int v . grad_x Q
    int qa = eb.a + (c == 0), qb = eb.b + (c == 1), qc = eb.c + (c == 2);
    const double id1 = inv_small(d + 1);
    double acc = hK * id1 * GM[(size_t)idx3(qa, qb, qc) * nK + col];
    if (d == 0) return acc;
    // curl part: R = -(grad m_b x e_c)/(d+1), components R_i = -(1/(d+1)) eps(i,j,c) d_j m_b
    for (int i = 0; i < 3; ++i)
      for (int jd = 0; jd < 3; ++jd) {
        if (i == jd || jd == c || i == c) continue;
        int eps = ((i + 1) % 3 == jd) ? 1 : -1;   // eps(i, jd, c) with c the third index
        int pj = jd == 0 ? eb.a : (jd == 1 ? eb.b : eb.c);
        if (pj == 0) continue;
        int ra = eb.a - (jd == 0), rb = eb.b - (jd == 1), rc = eb.c - (jd == 2);
        int rb_idx = idx3(ra, rb, rc);
        double coef = -(double)(eps * pj) * id1;
        double mom;
        if (d - 1 <= K - 3) mom = d4(col, rb_idx, i);
        else mom = use_enh ? enh(col, rb_idx, i) : 0.0;
        acc += coef * mom;
      }
    return acc;
  }

  VB_HD bool build(double nu, double* Aout, double* Bout, double* P0out, double* WMout = nullptr) {
    geometry();
    for (int g = ex.tid; g < S::NP1; g += ex.nt) sh.bndm[g] = 0.0;
    ex.sync();
    volume_moments();
    if (WMout)
      for (int a = ex.tid; a < S::NP0; a += ex.nt) WMout[a] = sh.mu[a];   // int_K m_a
    bool ok = volume_systems();
    for (int f = 0; f < R.nf; ++f) ok = face(f) && ok;
    const double hK = sh.hK, vol = sh.vol;
    const double ihK = 1.0 / hK, ivol = 1.0 / vol;
    for (int f = ex.tid; f < R.nf; f += ex.nt) sh.ifarea[f] = 1.0 / sh.farea[f];
    ex.sync();
    // (1) divergence: mom rows -> DIV = Minv0 mom
    for (int idx = ex.tid; idx < S::NP0 * nK; idx += ex.nt) {
      int g = idx / nK, col = idx % nK;
      double v = 0.0;
      // mom row 0 : sum_f sgn |f| (normal D3, b = 0)
      double m0 = 0.0;
      if (col >= off_f && col < off_4) {
        int r = col - off_f;
        int f = r / (3 * S::NFM), b = (r / 3) % S::NFM, t = r % 3;
        if (b == 0 && t == 0) m0 = R.fsign[f] * sh.farea[f];
      }
      v += sh.Minv0[g * S::NP0 + 0] * m0;
      if (col >= off_5) v += sh.Minv0[g * S::NP0 + (col - off_5 + 1)] * vol;
      DIV[idx] = v;
    }
    ex.sync();
    // (2) GM[a] = int v . grad_x m_a  for a in P_{k+1}
    for (int idx = ex.tid; idx < S::NP2 * nK; idx += ex.nt) {
      int a = idx / nK, col = idx % nK;
      // -int div v m_a
      double v = 0.0;
      for (int g = 0; g < S::NP0; ++g) v -= mass(g, a) * DIV[(size_t)g * nK + col];
      for (int c = 0; c < 3; ++c) v += bnd(col, c, a, c);
      GM[idx] = v;
    }
    ex.sync();
    // note: GM holds int v.grad_x Q when multiplied by ... (grad_x m_a = (1/h) grad_xi m_a)
    // vecmom uses h * int v . grad_x Q with Q in xi; int v.grad_x m_a as computed
    // above is int v . grad_x (m_a(xi)) = (1/h) int v . grad_xi m_a -- consistent.
    // (3) low moments (degree <= k-2), no enhancement
    for (int idx = ex.tid; idx < 3 * S::NL * nK; idx += ex.nt) {
      int c = idx / (S::NL * nK), r = idx % (S::NL * nK);
      int b = r / nK, col = r % nK;
      VML[idx] = vecmom(col, c, b, false);
    }
    ex.sync();
    // (4) Pi^nabla_k : G c = rhs
    {
      double* Gm = sh.big;
      for (int idx = ex.tid; idx < S::NP1 * S::NP1; idx += ex.nt) {
        const int p = idx / S::NP1, q = idx % S::NP1;
        double v = 0.0;
        if (p == 0) v = sh.bndm[q];
        else {
          const Exp3 ep = T.e3[p], eq = T.e3[q];
          if (ep.a && eq.a) v += ep.a * eq.a * mu(ep.a + eq.a - 2, ep.b + eq.b, ep.c + eq.c);
          if (ep.b && eq.b) v += ep.b * eq.b * mu(ep.a + eq.a, ep.b + eq.b - 2, ep.c + eq.c);
          if (ep.c && eq.c) v += ep.c * eq.c * mu(ep.a + eq.a, ep.b + eq.b, ep.c + eq.c - 2);
          v /= hK * hK;
        }
        Gm[idx] = v;
      }
      ex.sync();
      if (ex.tid < 32) ok = small_inverse_warp(Gm, sh.Ginv, S::NP1, ex.tid) && ok;
    }
    ex.sync();
    // rhs into VMH (temporary), then PiN = Ginv rhs
    for (int idx = ex.tid; idx < 3 * S::NP1 * nK; idx += ex.nt) {
      int c = idx / (S::NP1 * nK), r = idx % (S::NP1 * nK);
      int a = r / nK, col = r % nK;
      double v;
      if (a == 0) {
        v = bnd(col, c, 0, -1);
      } else {
        const Exp3 ea = T.e3[a];
        v = 0.0;
        // -int v_c Lap m_a, Lap_x m_a = (1/h^2) sum_j a_j (a_j - 1) m_{a - 2 e_j}
        if (ea.a >= 2) v -= ea.a * (ea.a - 1) * VML[((size_t)c * S::NL + idx3(ea.a - 2, ea.b, ea.c)) * nK + col];
        if (ea.b >= 2) v -= ea.b * (ea.b - 1) * VML[((size_t)c * S::NL + idx3(ea.a, ea.b - 2, ea.c)) * nK + col];
        if (ea.c >= 2) v -= ea.c * (ea.c - 1) * VML[((size_t)c * S::NL + idx3(ea.a, ea.b, ea.c - 2)) * nK + col];
        v *= ihK * ihK;
        // + int_dK v_c grad m_a . n = (1/h) sum_j a_j int_dK v_c m_{a-e_j} n_j
        if (ea.a) v += ea.a * ihK * bnd(col, c, idx3(ea.a - 1, ea.b, ea.c), 0);
        if (ea.b) v += ea.b * ihK * bnd(col, c, idx3(ea.a, ea.b - 1, ea.c), 1);
        if (ea.c) v += ea.c * ihK * bnd(col, c, idx3(ea.a, ea.b, ea.c - 1), 2);
      }
      VMH[idx] = v;
    }
    ex.sync();
    for (int idx = ex.tid; idx < 3 * S::NP1 * nK; idx += ex.nt) {
      int c = idx / (S::NP1 * nK), r = idx % (S::NP1 * nK);
      int a = r / nK, col = r % nK;
      double acc = 0.0;
      for (int g = 0; g < S::NP1; ++g) acc += sh.Ginv[a * S::NP1 + g] * VMH[((size_t)c * S::NP1 + g) * nK + col];
      PiN[idx] = acc;
    }
    ex.sync();
    // (5) Pi^0_{k-1} grad v, symmetrized: Rs_ij = (rhs_ij + rhs_ji)/2, E_ij = Minv0 Rs_ij
    //     rhs_ij[a] = -(a_j/h) int v_i m_{a-e_j} + int_dK v_i m_a n_j
    for (int idx = ex.tid; idx < 6 * S::NP0 * nK; idx += ex.nt) {
      int pr = idx / (S::NP0 * nK), r = idx % (S::NP0 * nK);
      int a = r / nK, col = r % nK;
      const int PI[6] = {0, 1, 2, 0, 0, 1}, PJ[6] = {0, 1, 2, 1, 2, 2};
      int i = PI[pr], j = PJ[pr];
      const Exp3 ea = T.e3[a];
      double v = 0.0;
      for (int s = 0; s < 2; ++s) {
        int ii = s ? j : i, jj = s ? i : j;
        int pj = jj == 0 ? ea.a : (jj == 1 ? ea.b : ea.c);
        if (pj > 0) {
          int bidx = idx3(ea.a - (jj == 0), ea.b - (jj == 1), ea.c - (jj == 2));
          v -= pj * ihK * VML[((size_t)ii * S::NL + bidx) * nK + col];
        }
        v += bnd(col, ii, a, jj);
      }
      Rs[idx] = 0.5 * v;
    }
    ex.sync();
    for (int idx = ex.tid; idx < 6 * S::NP0 * nK; idx += ex.nt) {
      int pr = idx / (S::NP0 * nK), r = idx % (S::NP0 * nK);
      int a = r / nK, col = r % nK;
      double acc = 0.0;
      for (int g = 0; g < S::NP0; ++g) acc += sh.Minv0[a * S::NP0 + g] * Rs[((size_t)pr * S::NP0 + g) * nK + col];
      E[idx] = acc;
    }
    ex.sync();
    // (6) DOFs of the [P_k]^3 basis: Dm[row][c*NP1 + a]
    const int nb = 3 * S::NP1;
    for (int idx = ex.tid; idx < nK * nb; idx += ex.nt) {
      int row = idx / nb, cb = idx % nb;
      int c = cb / S::NP1, a = cb % S::NP1;
      const Exp3 ea = T.e3[a];
      double v = 0.0;
      const double hi = ihK;
      if (row < off_e) {
        if (row % 3 == c) {
          const double* X = sh.X[row / 3];
          v = ipow((X[0] - sh.xK[0]) * hi, ea.a) * ipow((X[1] - sh.xK[1]) * hi, ea.b) * ipow((X[2] - sh.xK[2]) * hi, ea.c);
        }
      } else if (row < off_f) {
        int r = row - off_e;
        int le = r / (3 * (K - 1)), jj = (r / 3) % (K - 1), cc = r % 3;
        if (cc == c) {
          // edge from its lower vertex: vertices are stored sorted, so locate them
          int a0 = R.edge_a[le], b0 = R.edge_b[le];
          const double *PA = nullptr, *PB = nullptr;
          for (int q = 0; q < R.nv; ++q) {
            if (R.vert[q] == a0) PA = sh.X[q];
            if (R.vert[q] == b0) PB = sh.X[q];
          }
          double t = T.gl[jj];
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = PA[d] + t * (PB[d] - PA[d]);
          v = ipow((x[0] - sh.xK[0]) * hi, ea.a) * ipow((x[1] - sh.xK[1]) * hi, ea.b) * ipow((x[2] - sh.xK[2]) * hi, ea.c);
        }
      } else if (row < off_4) {
        int r = row - off_f;
        int f = r / (3 * S::NFM), b = (r / 3) % S::NFM, t = r % 3;
        double wv = t == 0 ? sh.fn[f][c] : (t == 1 ? sh.ft1[f][c] : sh.ft2[f][c]);
        // (1/|f|) int_f m3_a m2_b from the face moments kept by face(f)
        v = wv * FM[((size_t)f * S::NP1 + a) * S::NFM + b] * sh.ifarea[f];
      } else if (row < off_5) {
        int jcol = row - off_4;
        // generator number g (kept ones in order, the dropped one skipped)
        int g = jcol;
        if (K == 4 && g >= 11) g += 1;
        int bb = g / 3, i = g % 3;
        // (1/|K|) int m_a e_c . (xi ^ (m_bb e_i)) = (1/|K|) int m_a eps(c,j,i) xi_j m_bb
        const Exp3 eb = T.e3[bb];
        for (int jd = 0; jd < 3; ++jd) {
          if (c == jd || jd == i || c == i) continue;
          int eps = ((c + 1) % 3 == jd) ? 1 : -1;
          v += eps * mu(ea.a + eb.a + (jd == 0), ea.b + eb.b + (jd == 1), ea.c + eb.c + (jd == 2));
        }
        v *= ivol;
      } else {
        int al = row - off_5 + 1;
        // (1/|K|) int div(m_a e_c) m_al = (1/|K|) (p_c/h) int m_{a-e_c} m_al
        int pc = c == 0 ? ea.a : (c == 1 ? ea.b : ea.c);
        if (pc > 0) {
          const Exp3 el = T.e3[al];
          v = pc * hi * mu(ea.a - (c == 0) + el.a, ea.b - (c == 1) + el.b, ea.c - (c == 2) + el.c) * ivol;
        }
      }
      Dm[idx] = v;
    }
    ex.sync();
    // (7) consistency Ac = sum_ij Rs_ij^T E_ij (off-diagonal pairs twice), into Pm[nK*nK ..]
    double* Ac = Pm + (size_t)nK * nK;
    // (symmetric: the upper triangle is formed, rows p and nK-1-p paired,
    // and mirrored)
    for (int idx = ex.tid; idx < ((nK + 1) / 2) * (nK + 1); idx += ex.nt) {
      const int p = idx / (nK + 1), j = idx % (nK + 1);
      int r, c;
      if (j < nK - p) { r = p; c = p + j; }
      else { r = nK - 1 - p; c = r + (j - (nK - p)); if (r == p) continue; }
      double acc = 0.0;
      for (int pr = 0; pr < 6; ++pr) {
        double w = pr < 3 ? 1.0 : 2.0;
        double s = 0.0;
        for (int g = 0; g < S::NP0; ++g)
          s += Rs[((size_t)pr * S::NP0 + g) * nK + r] * E[((size_t)pr * S::NP0 + g) * nK + c];
        acc += w * s;
      }
      Ac[(size_t)r * nK + c] = acc;
      Ac[(size_t)c * nK + r] = acc;
    }
    ex.sync();
    // (8)-(9) A = nu (Ac + P^T diag(s) P), s_i = max(Ac_ii, h_K), with
    // P = I - X, X = Dm PiN of rank nb, through the low-rank expansion
    //   P^T S P = S - F PiN - (F PiN)^T + PiN^T W PiN,  F = S Dm, W = Dm^T F
    // (F: nK x nb and G = W PiN: nb x nK, row-major, in the Pm scratch)
    double* F = Pm;
    double* W = Pm + (size_t)nK * nb;
    double* G = W + (size_t)nb * nb;
    for (int idx = ex.tid; idx < nK * nb; idx += ex.nt) {
      const int r = idx / nb;
      const double sr = Ac[(size_t)r * nK + r];
      F[idx] = (sr > hK ? sr : hK) * Dm[idx];
    }
    ex.sync();
    for (int idx = ex.tid; idx < nb * nb; idx += ex.nt) {
      const int a = idx / nb, bq = idx % nb;
      double acc = 0.0;
      for (int q = 0; q < nK; ++q) acc += Dm[(size_t)q * nb + a] * F[(size_t)q * nb + bq];
      W[idx] = acc;
    }
    ex.sync();
    // G <- W PiN - F^T: then (P^T S P - S)[r][c] = sum_q PiN[q][r] G[q][c] - F[r][q] PiN[q][c]
    for (int idx = ex.tid; idx < nb * nK; idx += ex.nt) {
      const int a = idx / nK, c = idx % nK;
      double acc = 0.0;
      for (int bq = 0; bq < nb; ++bq) acc += W[(size_t)a * nb + bq] * PiN[(size_t)bq * nK + c];
      G[idx] = acc - F[(size_t)c * nb + a];
    }
    ex.sync();
    // upper triangle only, rows p and nK-1-p paired (nK+1 entries per pair)
    for (int idx = ex.tid; idx < ((nK + 1) / 2) * (nK + 1); idx += ex.nt) {
      const int p = idx / (nK + 1), j = idx % (nK + 1);
      int r, c;
      if (j < nK - p) { r = p; c = p + j; }
      else { r = nK - 1 - p; c = r + (j - (nK - p)); if (r == p) continue; }
      double acc = 0.0;
      if (r == c) {
        const double sr = Ac[(size_t)r * nK + r];
        acc = sr > hK ? sr : hK;
      }
      const double* fr = F + (size_t)r * nb;
      for (int q = 0; q < nb; ++q) acc += PiN[(size_t)q * nK + r] * G[(size_t)q * nK + c] - fr[q] * PiN[(size_t)q * nK + c];
      double v = nu * (Ac[(size_t)r * nK + c] + acc);
      Aout[(size_t)r * nK + c] = v;
      Aout[(size_t)c * nK + r] = v;
    }
    // (10) B_K rows: row 0 flux, rows a >= 1: |K| on D5
    for (int idx = ex.tid; idx < S::NP0 * nK; idx += ex.nt) {
      int a = idx / nK, col = idx % nK;
      double v = 0.0;
      if (a == 0) {
        if (col >= off_f && col < off_4) {
          int r = col - off_f;
          int f = r / (3 * S::NFM), b = (r / 3) % S::NFM, t = r % 3;
          if (b == 0 && t == 0) v = R.fsign[f] * sh.farea[f];
        }
      } else if (col == off_5 + a - 1) {
        v = vol;
      }
      Bout[idx] = v;
    }
    ex.sync();
    // (11) Pi^0_k : VMH[c][a] = int v . m_a e_c (with enhancement), P0 = Minv1 VMH
    for (int idx = ex.tid; idx < 3 * S::NP1 * nK; idx += ex.nt) {
      int c = idx / (S::NP1 * nK), r = idx % (S::NP1 * nK);
      int a = r / nK, col = r % nK;
      VMH[idx] = vecmom(col, c, a, true);
    }
    ex.sync();
    for (int idx = ex.tid; idx < 3 * S::NP1 * nK; idx += ex.nt) {
      int c = idx / (S::NP1 * nK), r = idx % (S::NP1 * nK);
      int a = r / nK, col = r % nK;
      double acc = 0.0;
      for (int g = 0; g < S::NP1; ++g) acc += sh.Minv1[a * S::NP1 + g] * VMH[((size_t)c * S::NP1 + g) * nK + col];
      P0out[idx] = acc;
    }
    ex.sync();
    return ok;
  }
};

}  // namespace vb

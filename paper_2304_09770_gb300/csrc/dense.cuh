// Batched dense FP64 linear algebra for the adaptive coarse space (Sec. 6):
// one small symmetric matrix per macro face (n up to about a thousand),
// column-major with leading dimension n, addressed through DenseItem
// offsets.  GEMM tiles spread over many CTAs; the factorizations and the
// eigen-solver steps run one CTA per face, with the matrix in global memory
// and the vectors of the current step in shared memory.
#pragma once
#include "launch.h"

namespace vb {

struct DenseItem {
  int n;
  int64_t a, b, c;   // offsets of the operands of this item (meaning per kernel)
};
struct GemmTask {
  int item, ti, tj;
};

// C = alpha op(A) B + beta C per item (n x n, column-major), op(A) = A or A^T;
// 64 x 64 output tiles, 256 threads with 4 x 4 outputs each, k staged by 16
struct KBatchGemm {
  const double* A;
  const double* Bm;
  double* C;
  const DenseItem* items;
  const GemmTask* tasks;
  int transA;
  double alpha, beta;
  __device__ void operator()(const KExec& ex, int blk) const {
    const GemmTask tk = tasks[blk];
    const DenseItem it = items[tk.item];
    const int n = it.n, r0 = tk.ti * 64, c0 = tk.tj * 64;
    const double* a = A + it.a;
    const double* bm = Bm + it.b;
    double* c = C + it.c;
    double* As = ex.smem;            // [16][65]: As[kk*65 + m] = op(A)(r0+m, k0+kk)
    double* Bs = ex.smem + 16 * 65;  // [16][65]: Bs[kk*65 + j] = B(k0+kk, c0+j)
    const int tx = ex.tid % 16, ty = ex.tid / 16;
    double acc[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += 16) {
      for (int idx = ex.tid; idx < 16 * 64; idx += ex.nt) {
        int m, kk;
        if (transA) { m = idx / 16; kk = idx % 16; } else { kk = idx / 64; m = idx % 64; }
        const int row = r0 + m, k = k0 + kk;
        double v = 0.0;
        if (row < n && k < n) v = transA ? a[(int64_t)row * n + k] : a[(int64_t)k * n + row];
        As[kk * 65 + m] = v;
        const int j = idx / 16, kb = idx % 16;
        const int col = c0 + j, kq = k0 + kb;
        Bs[kb * 65 + j] = (col < n && kq < n) ? bm[(int64_t)col * n + kq] : 0.0;
      }
      ex.sync();
#pragma unroll 4
      for (int kk = 0; kk < 16; ++kk) {
        double av[4], bv[4];
        for (int i = 0; i < 4; ++i) av[i] = As[kk * 65 + ty * 4 + i];
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk * 65 + tx * 4 + j];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
      ex.sync();
    }
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tx * 4 + j;
      if (col >= n) continue;
      for (int i = 0; i < 4; ++i) {
        const int row = r0 + ty * 4 + i;
        if (row >= n) continue;
        double* cp = c + (int64_t)col * n + row;
        *cp = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *cp);
      }
    }
  }
};

// X <- (X + X^T) / 2 per item (matrix at offset a)
struct KSymmetrize {
  double* X;
  const DenseItem* items;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int n = it.n;
    double* x = X + it.a;
    for (int64_t idx = ex.tid; idx < (int64_t)n * n; idx += ex.nt) {
      const int j = (int)(idx / n), i = (int)(idx % n);
      if (i > j) {
        const double s = 0.5 * (x[(int64_t)j * n + i] + x[(int64_t)i * n + j]);
        x[(int64_t)j * n + i] = s;
        x[(int64_t)i * n + j] = s;
      }
    }
  }
};

// In-place Cholesky X = G G^T (lower, column-major) per item, strict upper
// part set to zero; a non-positive pivot sets *status = 1 and stops that item
struct KCholesky {
  double* X;
  const DenseItem* items;
  int* status;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int n = it.n;
    double* x = X + it.a;
    const int nw = ex.nt >> 5, w = ex.tid >> 5, lane = ex.tid & 31;
    for (int j = 0; j < n; ++j) {
      const double d = x[(int64_t)j * n + j];
      if (!(d > 0.0)) {
        if (ex.tid == 0) flag_error(status, 1);
        return;
      }
      const double s = sqrt(d), inv = 1.0 / s;
      ex.sync();
      for (int i = j + 1 + ex.tid; i < n; i += ex.nt) x[(int64_t)j * n + i] *= inv;
      if (ex.tid == 0) x[(int64_t)j * n + j] = s;
      ex.sync();
      for (int k = j + 1 + w; k < n; k += nw) {
        const double lk = x[(int64_t)j * n + k];
        double* col = x + (int64_t)k * n;
        const double* lj = x + (int64_t)j * n;
        for (int i = k + lane; i < n; i += 32) col[i] -= lj[i] * lk;
      }
      ex.sync();
    }
    for (int64_t idx = ex.tid; idx < (int64_t)n * n; idx += ex.nt) {
      const int j = (int)(idx / n), i = (int)(idx % n);
      if (i < j) x[idx] = 0.0;
    }
  }
};

// Householder tridiagonalization Q^T X Q = T of a symmetric item (full
// storage, overwritten): diagonal d[n], subdiagonal e[n-1]; reflector k
// (I - tau_k v v^T on rows k+1..n-1) kept in column k below the diagonal
// (entries k+1..n-1) and tau[k].  Offsets: matrix it.a, d and e at it.b
// (d: n values, e: n values), tau at it.c (n values).
struct KTridiag {
  double* X;
  double* DE;
  double* TAU;
  const DenseItem* items;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int n = it.n;
    double* x = X + it.a;
    double* d = DE + it.b;
    double* e = d + n;
    double* tau = TAU + it.c;
    double* v = ex.smem;          // [n]
    double* p = ex.smem + n;      // [n]
    double* red = ex.smem + 2 * n;   // [nt]
    for (int k = 0; k + 2 < n; ++k) {
      const int m = n - k - 1;
      double* xc = x + (int64_t)k * n + k + 1;   // column k below the diagonal
      double ss = 0.0;
      for (int i = ex.tid; i < m; i += ex.nt) {
        v[i] = xc[i];
        ss += v[i] * v[i];
      }
      ss = block_sum(ex, ss, red);
      const double x0 = v[0];
      const double nrm = sqrt(ss);
      if (ex.tid == 0) d[k] = x[(int64_t)k * n + k];
      if (nrm == 0.0) {
        if (ex.tid == 0) { e[k] = 0.0; tau[k] = 0.0; }
        ex.sync();
        continue;
      }
      const double beta = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - beta;
      const double t = -v0 / beta;            // tau with v scaled to v[0] = 1
      const double sc = 1.0 / v0;
      ex.sync();
      for (int i = ex.tid; i < m; i += ex.nt) {
        const double vi = i == 0 ? 1.0 : v[i] * sc;
        v[i] = vi;
        xc[i] = vi;
      }
      if (ex.tid == 0) { e[k] = beta; tau[k] = t; }
      ex.sync();
      // p = t A' v (A' the trailing block, rows/columns k+1..n-1)
      const double* ap = x + (int64_t)(k + 1) * n + k + 1;
      for (int i = ex.tid; i < m; i += ex.nt) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += ap[(int64_t)j * n + i] * v[j];
        p[i] = t * s;
      }
      ex.sync();
      double pv = 0.0;
      for (int i = ex.tid; i < m; i += ex.nt) pv += p[i] * v[i];
      pv = block_sum(ex, pv, red);
      const double K = 0.5 * t * pv;
      for (int i = ex.tid; i < m; i += ex.nt) p[i] -= K * v[i];   // w
      ex.sync();
      // A' -= v w^T + w v^T
      double* aw = x + (int64_t)(k + 1) * n + k + 1;
      for (int64_t idx = ex.tid; idx < (int64_t)m * m; idx += ex.nt) {
        const int j = (int)(idx / m), i = (int)(idx % m);
        aw[(int64_t)j * n + i] -= v[i] * p[j] + p[i] * v[j];
      }
      ex.sync();
    }
    if (ex.tid == 0) {
      if (n >= 2) {
        d[n - 2] = x[(int64_t)(n - 2) * n + n - 2];
        e[n - 2] = x[(int64_t)(n - 2) * n + n - 1];
        tau[n - 2] = 0.0;
      }
      d[n - 1] = x[(int64_t)(n - 1) * n + n - 1];
      tau[n - 1] = 0.0;
      e[n - 1] = 0.0;
    }
  }
};

// number of eigenvalues of the tridiagonal (d, e) below x (Sturm sequence)
__device__ inline int sturm_count(const double* d, const double* e, int n, double x, double tiny) {
  int c = 0;
  double q = d[0] - x;
  for (int i = 0;; ++i) {
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++c;
    if (i + 1 >= n) break;
    q = d[i + 1] - x - e[i] * e[i] / q;
  }
  return c;
}

// Eigenpairs of the tridiagonal (d, e) with eigenvalue above theta: the
// count (capped at maxsel; *count_out holds the uncapped number), the
// eigenvalues by bisection (largest first) and eigenvectors by inverse
// iteration with Gram-Schmidt against the vectors already found, then
// back-transformed with the reflectors (eigenvectors of the original
// matrix).  Offsets: reflectors in the matrix at it.a, d/e at it.b, tau at
// it.c; outputs per item index blk: lam[blk*maxsel + s], Y[yoff[blk] + s*n].
struct KTridiagEig {
  const double* X;
  const double* DE;
  const double* TAU;
  const DenseItem* items;
  double theta;
  int maxsel;
  int* count_out;
  double* lam;
  double* Y;
  const int64_t* yoff;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int n = it.n;
    const double* x = X + it.a;
    const double* d = DE + it.b;
    const double* e = d + n;
    const double* tau = TAU + it.c;
    double* ds = ex.smem;             // [n] diagonal
    double* es = ds + n;              // [n] off-diagonal
    double* lu = es + n;              // [n] multipliers l_i
    double* uu = lu + n;              // [n] pivots u_i
    double* red = uu + n;             // [nt]
    double* sh = red + ex.nt;         // [maxsel] eigenvalues
    for (int i = ex.tid; i < n; i += ex.nt) {
      ds[i] = d[i];
      es[i] = e[i];
    }
    ex.sync();
    // Gershgorin bounds and the scale of T
    double lo = 1e300, hi = -1e300, sc = 0.0;
    for (int i = ex.tid; i < n; i += ex.nt) {
      const double r = (i > 0 ? fabs(es[i - 1]) : 0.0) + (i + 1 < n ? fabs(es[i]) : 0.0);
      lo = fmin(lo, ds[i] - r);
      hi = fmax(hi, ds[i] + r);
      sc = fmax(sc, fabs(ds[i]) + r);
    }
    red[ex.tid] = lo;
    ex.sync();
    for (int s = ex.nt / 2; s > 0; s >>= 1) {
      if (ex.tid < s) red[ex.tid] = fmin(red[ex.tid], red[ex.tid + s]);
      ex.sync();
    }
    lo = red[0];
    ex.sync();
    red[ex.tid] = hi;
    ex.sync();
    for (int s = ex.nt / 2; s > 0; s >>= 1) {
      if (ex.tid < s) red[ex.tid] = fmax(red[ex.tid], red[ex.tid + s]);
      ex.sync();
    }
    hi = red[0];
    ex.sync();
    red[ex.tid] = sc;
    ex.sync();
    for (int s = ex.nt / 2; s > 0; s >>= 1) {
      if (ex.tid < s) red[ex.tid] = fmax(red[ex.tid], red[ex.tid + s]);
      ex.sync();
    }
    sc = fmax(red[0], 1e-300);
    ex.sync();
    const double tiny = 1e-300;
    const int below = sturm_count(ds, es, n, theta, tiny);
    const int total = n - below;
    const int m = total < maxsel ? total : maxsel;
    if (ex.tid == 0) count_out[blk] = total;
    // eigenvalue index n-1-s (descending) by bisection, one thread each
    for (int s = ex.tid; s < m; s += ex.nt) {
      const int idx = n - 1 - s;
      double a = fmax(theta, lo), b = hi;
      for (int iter = 0; iter < 200 && b - a > 4e-16 * fmax(fabs(a), fabs(b)); ++iter) {
        const double mid = 0.5 * (a + b);
        if (sturm_count(ds, es, n, mid, tiny) > idx) b = mid; else a = mid;
      }
      sh[s] = 0.5 * (a + b);
      lam[(int64_t)blk * maxsel + s] = sh[s];
    }
    ex.sync();
    double* Yb = Y + yoff[blk];
    const double ptiny = 1e-14 * sc;
    for (int s = 0; s < m; ++s) {
      const double mu = sh[s];
      double* y = Yb + (int64_t)s * n;
      // T - mu I = L U without pivoting, tiny pivots replaced by +-ptiny
      if (ex.tid == 0) {
        double u = ds[0] - mu;
        if (fabs(u) < ptiny) u = u < 0.0 ? -ptiny : ptiny;
        uu[0] = u;
        for (int i = 1; i < n; ++i) {
          const double l = es[i - 1] / uu[i - 1];
          lu[i] = l;
          u = ds[i] - mu - l * es[i - 1];
          if (fabs(u) < ptiny) u = u < 0.0 ? -ptiny : ptiny;
          uu[i] = u;
        }
      }
      for (int i = ex.tid; i < n; i += ex.nt) y[i] = 1.0 + 0.001 * (double)((i * 7 + s * 13) % 17);
      ex.sync();
      for (int iter = 0; iter < 3; ++iter) {
        if (ex.tid == 0) {
          for (int i = 1; i < n; ++i) y[i] -= lu[i] * y[i - 1];
          y[n - 1] /= uu[n - 1];
          for (int i = n - 2; i >= 0; --i) y[i] = (y[i] - es[i] * y[i + 1]) / uu[i];
        }
        ex.sync();
        // orthogonalize against the vectors found so far, then normalize
        for (int q = 0; q < s; ++q) {
          const double* yq = Yb + (int64_t)q * n;
          double dt = 0.0;
          for (int i = ex.tid; i < n; i += ex.nt) dt += yq[i] * y[i];
          dt = block_sum(ex, dt, red);
          for (int i = ex.tid; i < n; i += ex.nt) y[i] -= dt * yq[i];
          ex.sync();
        }
        double nn = 0.0;
        for (int i = ex.tid; i < n; i += ex.nt) nn += y[i] * y[i];
        nn = block_sum(ex, nn, red);
        const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int i = ex.tid; i < n; i += ex.nt) y[i] *= inv;
        ex.sync();
      }
    }
    // back-transform: y <- H_0 H_1 ... H_{n-3} y, one warp per vector
    const int nw = ex.nt >> 5, w = ex.tid >> 5, lane = ex.tid & 31;
    for (int s = w; s < m; s += nw) {
      double* y = Yb + (int64_t)s * n;
      for (int k = n - 3; k >= 0; --k) {
        const double t = tau[k];
        if (t == 0.0) continue;
        const double* vk = x + (int64_t)k * n + k + 1;
        double dt = 0.0;
        for (int i = lane; i < n - k - 1; i += 32) dt += vk[i] * y[k + 1 + i];
        for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
        dt *= t;
        for (int i = lane; i < n - k - 1; i += 32) y[k + 1 + i] -= dt * vk[i];
        __syncwarp();
      }
    }
  }
};

// out_s = L y_s (L lower triangular at it.a) then row_s = B out_s (B at
// it.b), for the selected vectors of each item; rows written over Y
struct KConstraintRows {
  const double* Lm;
  const double* Bm;
  double* Y;
  const int64_t* yoff;
  const DenseItem* items;
  const int* count;
  int maxsel;
  __device__ void operator()(const KExec& ex, int blk) const {
    const DenseItem it = items[blk];
    const int n = it.n;
    const int m = count[blk] < maxsel ? count[blk] : maxsel;
    const double* L = Lm + it.a;
    const double* B = Bm + it.b;
    double* t = ex.smem;   // [n]
    for (int s = 0; s < m; ++s) {
      double* y = Y + yoff[blk] + (int64_t)s * n;
      for (int i = ex.tid; i < n; i += ex.nt) {
        double acc = 0.0;
        for (int j = 0; j <= i; ++j) acc += L[(int64_t)j * n + i] * y[j];
        t[i] = acc;
      }
      ex.sync();
      for (int i = ex.tid; i < n; i += ex.nt) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += B[(int64_t)j * n + i] * t[j];
        y[i] = acc;
      }
      ex.sync();
    }
  }
};

}  // namespace vb

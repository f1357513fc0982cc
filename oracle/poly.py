"""Scaled monomials, coefficient-space polynomial algebra and quadrature.

Test infrastructure only (see ``oracle/__init__.py``).

Monomial order: graded by total degree; inside a degree, lexicographically
descending in the first exponent, then the second.  In 3D degree 1 is
(x, y, z); in 2D degree 1 is (s, t).
"""
import numpy as np
from functools import lru_cache


@lru_cache(maxsize=None)
def exps3(n):
    out = []
    for d in range(n + 1):
        for a in range(d, -1, -1):
            for b in range(d - a, -1, -1):
                out.append((a, b, d - a - b))
    return tuple(out)


@lru_cache(maxsize=None)
def exps2(n):
    out = []
    for d in range(n + 1):
        for a in range(d, -1, -1):
            out.append((a, d - a))
    return tuple(out)


def dim3(n):
    return 0 if n < 0 else (n + 1) * (n + 2) * (n + 3) // 6


def dim2(n):
    return 0 if n < 0 else (n + 1) * (n + 2) // 2


@lru_cache(maxsize=None)
def index3(n):
    return {e: i for i, e in enumerate(exps3(n))}


@lru_cache(maxsize=None)
def index2(n):
    return {e: i for i, e in enumerate(exps2(n))}


@lru_cache(maxsize=None)
def _earr3(n):
    return np.array(exps3(n), dtype=np.int64).reshape(-1, 3)


@lru_cache(maxsize=None)
def _earr2(n):
    return np.array(exps2(n), dtype=np.int64).reshape(-1, 2)


def _powers(x, p):
    """x [P] -> [P, p+1] with columns x^0..x^p."""
    out = np.ones((len(x), p + 1))
    for i in range(1, p + 1):
        out[:, i] = out[:, i - 1] * x
    return out


def mono3(n, xi):
    """Values of all 3D monomials of degree <= n at points xi [P,3] -> [P, dim3(n)]."""
    xi = np.atleast_2d(xi)
    E = _earr3(n)
    px, py, pz = (_powers(xi[:, j], n) for j in range(3))
    return px[:, E[:, 0]] * py[:, E[:, 1]] * pz[:, E[:, 2]]


def mono2(n, st):
    st = np.atleast_2d(st)
    E = _earr2(n)
    ps, pt = _powers(st[:, 0], n), _powers(st[:, 1], n)
    return ps[:, E[:, 0]] * pt[:, E[:, 1]]


def dmono3(n, xi, j):
    """d/dxi_j of all monomials of degree <= n at points xi."""
    xi = np.atleast_2d(xi)
    E = _earr3(n).copy()
    coef = E[:, j].astype(np.float64)
    E[:, j] = np.maximum(E[:, j] - 1, 0)
    px, py, pz = (_powers(xi[:, i], n) for i in range(3))
    return coef[None, :] * px[:, E[:, 0]] * py[:, E[:, 1]] * pz[:, E[:, 2]]


def dmono2(n, st, j):
    st = np.atleast_2d(st)
    E = _earr2(n).copy()
    coef = E[:, j].astype(np.float64)
    E[:, j] = np.maximum(E[:, j] - 1, 0)
    ps, pt = _powers(st[:, 0], n), _powers(st[:, 1], n)
    return coef[None, :] * ps[:, E[:, 0]] * pt[:, E[:, 1]]


# ---- coefficient-space operators (3D), degree-n source -> degree-m target ----

def op_mul3(n, i):
    """Multiplication by xi_i: P_n -> P_{n+1} as a matrix [dim3(n+1), dim3(n)]."""
    tgt = index3(n + 1)
    M = np.zeros((dim3(n + 1), dim3(n)))
    for c, e in enumerate(exps3(n)):
        ee = list(e)
        ee[i] += 1
        M[tgt[tuple(ee)], c] = 1.0
    return M


def op_d3(n, i):
    """d/dxi_i: P_n -> P_{n-1} as a matrix [dim3(n-1), dim3(n)]."""
    M = np.zeros((dim3(n - 1), dim3(n)))
    if n == 0:
        return M
    tgt = index3(n - 1)
    for c, e in enumerate(exps3(n)):
        if e[i] > 0:
            ee = list(e)
            ee[i] -= 1
            M[tgt[tuple(ee)], c] = e[i]
    return M


def op_lap3(n):
    """Laplacian in xi: P_n -> P_{n-2} (embedded in P_{max(n-2,0)})."""
    m = max(n - 2, 0)
    M = np.zeros((dim3(m), dim3(n)))
    for i in range(3):
        D = op_d3(n - 1, i) @ op_d3(n, i) if n >= 2 else np.zeros((dim3(m), dim3(n)))
        M += D[:dim3(m), :]
    return M


def op_lap2(n, G=None):
    """sum_pq G_pq d_p d_q (the Laplacian for G = I): P_n -> P_{n-2}."""
    G = np.eye(2) if G is None else G
    m = max(n - 2, 0)
    M = np.zeros((dim2(m), dim2(n)))
    tgt = index2(m)
    for c, (a, b) in enumerate(exps2(n)):
        if a >= 2:
            M[tgt[(a - 2, b)], c] += G[0, 0] * a * (a - 1)
        if a >= 1 and b >= 1:
            M[tgt[(a - 1, b - 1)], c] += 2.0 * G[0, 1] * a * b
        if b >= 2:
            M[tgt[(a, b - 2)], c] += G[1, 1] * b * (b - 1)
    return M


def embed3(n, m):
    """Injection P_n -> P_m (m >= n)."""
    E = np.zeros((dim3(m), dim3(n)))
    E[:dim3(n), :dim3(n)] = np.eye(dim3(n))
    return E


def degree_mask3(n, degs):
    return np.array([sum(e) in degs for e in exps3(n)])


def cross_xi(n):
    """Operator R -> xi ^ R from [P_n]^3 to [P_{n+1}]^3 (component-major blocks)."""
    X = [op_mul3(n, i) for i in range(3)]
    N1, N0 = dim3(n + 1), dim3(n)
    C = np.zeros((3 * N1, 3 * N0))
    # (xi ^ R)_0 = xi_1 R_2 - xi_2 R_1, etc.
    C[0:N1, 2 * N0:3 * N0] += X[1]
    C[0:N1, 1 * N0:2 * N0] -= X[2]
    C[N1:2 * N1, 0:N0] += X[2]
    C[N1:2 * N1, 2 * N0:3 * N0] -= X[0]
    C[2 * N1:3 * N1, 1 * N0:2 * N0] += X[0]
    C[2 * N1:3 * N1, 0:N0] -= X[1]
    return C


def grad_op(n):
    """Operator Q -> grad_xi Q from P_{n+1} to [P_n]^3."""
    return np.vstack([op_d3(n + 1, i) for i in range(3)])


@lru_cache(maxsize=None)
def helmholtz_split(n):
    """For every vector monomial w = m_a e_c of degree <= n, a pair (Q, R)
    with w = grad_xi Q + xi ^ R, Q in P_{n+1} (no constant), R in [P_{n-1}]^3.

    Uses [P_n]^3 = grad P_{n+1} (+) xi ^ [P_{n-1}]^3.  The split of w is
    unique; R is taken of minimum norm (xi ^ R is what matters).
    Returns (Qc [dim3(n+1), 3 dim3(n)], Rc [3 dim3(n-1), 3 dim3(n)]).
    """
    G = grad_op(n)                       # [3 N_n, N_{n+1}]
    G = G[:, 1:]                          # drop the constant of Q
    if n >= 1:
        C = cross_xi(n - 1)              # [3 N_n, 3 N_{n-1}]
    else:
        C = np.zeros((3 * dim3(n), 0))
    L = np.hstack([G, C])
    W = np.eye(3 * dim3(n))
    sol, *_ = np.linalg.lstsq(L, W, rcond=None)
    res = L @ sol - W
    assert np.abs(res).max() < 1e-10, "Helmholtz-type split failed"
    Qc = np.zeros((dim3(n + 1), 3 * dim3(n)))
    Qc[1:, :] = sol[:G.shape[1], :]
    Rc = sol[G.shape[1]:, :]
    return Qc, Rc


# ---------------- quadrature ----------------

@lru_cache(maxsize=None)
def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


@lru_cache(maxsize=None)
def quad_tri(deg):
    """Collapsed Gauss rule on the triangle (0,0),(1,0),(0,1); exact to ``deg``."""
    n = (deg + 2) // 2 + 1
    u, wu = gauss01(n)
    v, wv = gauss01(n)
    U, V = np.meshgrid(u, v, indexing="ij")
    WU, WV = np.meshgrid(wu, wv, indexing="ij")
    x = U
    y = V * (1 - U)
    w = WU * WV * (1 - U)
    return np.stack([x.ravel(), y.ravel()], 1), w.ravel()


@lru_cache(maxsize=None)
def quad_tet(deg):
    """Collapsed Gauss rule on the unit tetrahedron; exact to ``deg``."""
    n = (deg + 3) // 2 + 1
    g, wg = gauss01(n)
    U, V, W = np.meshgrid(g, g, g, indexing="ij")
    WU, WV, WW = np.meshgrid(wg, wg, wg, indexing="ij")
    x = U
    y = V * (1 - U)
    z = W * (1 - U) * (1 - V)
    w = WU * WV * WW * (1 - U) ** 2 * (1 - V)
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1), w.ravel()


@lru_cache(maxsize=None)
def gauss_lobatto_interior(k):
    """The k-1 interior Gauss-Lobatto nodes on [0,1] (roots of P_k')."""
    if k <= 1:
        return np.zeros(0)
    c = np.zeros(k + 1)
    c[k] = 1.0
    r = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    return np.sort(0.5 * (np.real(r) + 1.0))

"""Pins of the oracle's VEM discretization against what the paper and the
mathematics fix: DOF counts printed in the paper, polynomial reproduction of
the projectors, exact consistency of a_h on [P_k]^3, rigid-body kernel, exact
divergence moments, the global patch test and the convergence rate."""
import os

import numpy as np
import pytest

from synth import cube_mesh
from oracle.vem import Topology, DofMap, System, build_element, total_dofs
from oracle.poly import mono3, dmono3, dim3, quad_tet

HERE = os.path.dirname(__file__)


def _golden_counts():
    rows = []
    for line in open(os.path.join(HERE, "golden", "paper_dof_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, k, nd = line.split()[:3]
        rows.append((int(n), int(k), int(nd)))
    return rows


@pytest.mark.parametrize("n,k,ndofs", _golden_counts())
def test_dof_counts_match_paper_tables(n, k, ndofs):
    topo = Topology(cube_mesh(n))
    assert total_dofs(topo.nV, topo.nEd, topo.nF, topo.nE, k) == ndofs


def test_element_dof_counts():
    # cube: 8 vertices, 12 edges, 6 faces; split hex: 18 edges, 12 faces
    for mesh, k, nk in ((cube_mesh(2), 2, 81), (cube_mesh(3, 0.2, 1), 2, 117),
                        (cube_mesh(3, 0.2, 1), 3, 252), (cube_mesh(3, 0.2, 1), 4, 432)):
        topo = Topology(mesh)
        dm = DofMap(topo, k)
        assert len(dm.element_dofs(topo, 0)) == nk


def _element(n, pert, k, e=0, seed=1):
    topo = Topology(cube_mesh(n, pert, seed))
    return build_element(topo, DofMap(topo, k), e, 1.0)


ELEMS = [(2, 0.0, 2, 0), (3, 0.2, 2, 13), (3, 0.2, 3, 13), (3, 0.2, 4, 13)]


@pytest.fixture(scope="module", params=ELEMS, ids=lambda p: f"n{p[0]}p{p[1]}k{p[2]}")
def element(request):
    n, pert, k, e = request.param
    return _element(n, pert, k, e)


def test_projectors_reproduce_polynomials(element):
    D = element.D
    I = np.eye(D.shape[1])
    tol = {2: 1e-12, 3: 1e-10, 4: 1e-8}[element.k]
    assert np.abs(element.PiN @ D - I).max() < tol
    assert np.abs(element.Pi0 @ D - I).max() < tol


def _exact_strain_gram(el):
    """int_K eps(p):eps(q) for the [P_k]^3 monomial basis, by direct quadrature
    of the exact monomial derivatives on the element's tetrahedra."""
    k, hK = el.k, el.hK
    Nk = dim3(k)
    pts, w = el.vq_pts, el.vq_w
    xi = (pts - el.xK) / hK
    dm = [dmono3(k, xi, j) / hK for j in range(3)]      # d m_a / dx_j
    nb = 3 * Nk
    G = np.zeros((len(pts), nb, 3, 3))
    for c in range(3):
        for j in range(3):
            G[:, c * Nk:(c + 1) * Nk, c, j] = dm[j]
    E = 0.5 * (G + np.swapaxes(G, 2, 3))
    return np.einsum("p,paij,pbij->ab", w, E, E)


def test_consistency_on_polynomials(element):
    D = element.D
    lhs = D.T @ element.A @ D
    rhs = _exact_strain_gram(element)
    tol = {2: 1e-11, 3: 1e-9, 4: 1e-6}[element.k]
    assert np.abs(lhs - rhs).max() < tol * max(1.0, np.abs(rhs).max())


def test_stiffness_kernel_is_rigid_motions(element):
    A = element.A
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    scale = ev[-1]
    nz = np.sum(np.abs(ev) < 1e-9 * scale)
    assert nz == 6
    assert ev[0] > -1e-9 * scale
    # rigid motions: constants and xi ^ e_c
    def rig(c, rot):
        def f(x):
            out = np.zeros((len(x), 3))
            if rot:
                e = np.zeros(3)
                e[c] = 1.0
                out[:] = np.cross((x - element.xK), e)
            else:
                out[:, c] = 1.0
            return out
        return f
    zero = lambda x: np.zeros(len(x))
    for c in range(3):
        for rot in (False, True):
            d = element.poly_dofs(rig(c, rot), zero)
            assert np.abs(element.A @ d).max() < 1e-9 * scale * np.abs(d).max()


def test_divergence_rows_exact(element):
    """B_K dofs(p) = int_K div p m_a for every p in [P_k]^3."""
    k, hK = element.k, element.hK
    Nk = dim3(k)
    xi = element.xi
    M = mono3(k - 1, xi)
    ref = np.zeros((dim3(k - 1), 3 * Nk))
    for c in range(3):
        dv = dmono3(k, xi, c) / hK
        ref[:, c * Nk:(c + 1) * Nk] = (M * element.vq_w[:, None]).T @ dv
    got = element.B @ element.D
    assert np.abs(got - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())


def _patch(n, pert, k, seed):
    """Non-homogeneous Dirichlet data of a solenoidal u in [P_k]^3 and
    p in P_{k-1}: the discrete solution must be the interpolant."""
    mesh = cube_mesh(n, pert, seed)
    b = np.array([1.0, 2.0, -3.0])
    u = lambda x: np.stack([x[:, 1] ** k + x[:, 2], x[:, 2] ** k + x[:, 0], x[:, 0] ** k + x[:, 1]], 1)
    lap = lambda x: np.stack([k * (k - 1) * x[:, 1] ** (k - 2), k * (k - 1) * x[:, 2] ** (k - 2),
                              k * (k - 1) * x[:, 0] ** (k - 2)], 1)
    f = lambda x: -0.5 * lap(x) - b            # -div(eps u) - grad p, div u = 0
    S = System(mesh, k, np.ones(n ** 3), f=f)
    uI = np.zeros(S.dm.nvel)
    for e, el in S.elements.items():
        uI[el.dofs] = el.poly_dofs(u, lambda x: np.zeros(len(x)))
    uh, ph = S.solve_direct(u_bnd=uI)
    npk = dim3(k - 1)
    pex = np.zeros(S.dm.npress)
    for e, el in S.elements.items():
        c = np.zeros(npk)
        c[0] = b @ el.xK
        c[1:4] = el.hK * b
        pex[e * npk:(e + 1) * npk] = c
    pex -= (S.wmean @ pex) / S.wmean.sum()
    return S, uh, uI, ph, pex


@pytest.mark.parametrize("n,pert,k", [(3, 0.2, 2), (2, 0.2, 3)])
def test_patch_test(n, pert, k):
    S, uh, uI, ph, pex = _patch(n, pert, k, seed=3)
    assert np.abs(uh - uI).max() < 1e-10 * np.abs(uI).max()
    assert np.abs(ph - pex).max() < 1e-8 * np.abs(pex).max()
    # discrete divergence-free: B u_h = 0 elementwise (flux row and D5 rows)
    assert np.abs(S.B @ uh).max() < 1e-11


def test_convergence_rate_cubic_solution():
    """u = (y^3, z^3, x^3) (solenoidal, degree k+1), p = 0, k = 2: the L2 error
    of Pi^0_k u_h decays like h^{k+1}."""
    u = lambda x: np.stack([x[:, 1] ** 3, x[:, 2] ** 3, x[:, 0] ** 3], 1)
    f = lambda x: -3.0 * np.stack([x[:, 1], x[:, 2], x[:, 0]], 1)
    errs = []
    for n in (2, 4):
        S = System(cube_mesh(n), 2, np.ones(n ** 3), f=f)
        uI = np.zeros(S.dm.nvel)
        for e, el in S.elements.items():
            uI[el.dofs] = el.poly_dofs(u, lambda x: np.zeros(len(x)))
        uh, _ = S.solve_direct(u_bnd=uI)
        e2 = n2 = 0.0
        Nk = dim3(2)
        for e, el in S.elements.items():
            c = el.Pi0 @ uh[el.dofs]
            M = mono3(2, el.xi)
            v = np.stack([M @ c[j * Nk:(j + 1) * Nk] for j in range(3)], 1)
            ue = u(el.vq_pts)
            e2 += el.vq_w @ np.sum((v - ue) ** 2, 1)
            n2 += el.vq_w @ np.sum(ue ** 2, 1)
        errs.append(np.sqrt(e2 / n2))
    rate = np.log(errs[0] / errs[1]) / np.log(2.0)
    assert 2.7 < rate < 3.3


def test_convergence_rates_manufactured_solution():
    """The manufactured solution of the benchmark load (u = curl psi,
    vanishing on the boundary, p = 0), k = 2, on 2^3, 4^3 and 8^3 cubes: the
    H^1 error of Pi^nabla_k u_h decays like h^k and the L^2 error of
    Pi^0_k u_h like h^{k+1} (convergence theorem, Sec. 3); the rates are
    taken between 4^3 and 8^3 (2^3 is still pre-asymptotic).  The gradient
    of u is taken by central differences of step 1e-6 (error ~1e-12)."""
    from oracle_cache import oracle_system
    from oracle.poly import dmono3
    from synth.fields import manufactured_u
    Nk = dim3(2)
    errs = []
    for n in (2, 4, 8):
        _, S = oracle_system("cube4_k2", n=n)
        uh, _ = S.solve_direct()
        e1 = n1 = e0 = n0 = 0.0
        d = 1e-6
        for e, el in S.elements.items():
            x = el.vq_pts
            ue = manufactured_u(x)
            gu = np.stack([(manufactured_u(x + d * np.eye(3)[j]) - manufactured_u(x - d * np.eye(3)[j])) / (2 * d)
                           for j in range(3)], 2)
            cN = el.PiN @ uh[el.dofs]
            g = np.stack([np.stack([dmono3(2, el.xi, j) @ cN[c * Nk:(c + 1) * Nk] / el.hK for j in range(3)], 1)
                          for c in range(3)], 1)
            e1 += el.vq_w @ np.sum((g - gu) ** 2, (1, 2))
            n1 += el.vq_w @ np.sum(gu ** 2, (1, 2))
            c0 = el.Pi0 @ uh[el.dofs]
            M = mono3(2, el.xi)
            v = np.stack([M @ c0[j * Nk:(j + 1) * Nk] for j in range(3)], 1)
            e0 += el.vq_w @ np.sum((v - ue) ** 2, 1)
            n0 += el.vq_w @ np.sum(ue ** 2, 1)
        errs.append((np.sqrt(e1 / n1), np.sqrt(e0 / n0)))
    assert errs[0][0] > errs[1][0] > errs[2][0] and errs[0][1] > errs[1][1] > errs[2][1]
    h1 = np.log(errs[1][0] / errs[2][0]) / np.log(2.0)
    l2 = np.log(errs[1][1] / errs[2][1]) / np.log(2.0)
    assert 1.8 < h1 < 2.2, h1
    assert 2.8 < l2 < 3.3, l2

"""Pins of the OCTA mesh family and of the oracle's VEM on its elements
(octahedra and cubes with one corner truncated: pentagonal faces).

* The DOF counts of octa_mesh(m) equal the counts the paper prints for its
  OCTA meshes (Tables 2 and 3, k = 2, 3, 4): this fixes the mesh family's
  vertex, edge, face and element counts.
* The mesh is a valid conforming polyhedral partition of the unit cube:
  closed elements, planar faces, volumes summing to 1, every interior face
  shared by two elements with opposite orientation.
* On both element shapes: the projectors reproduce [P_k]^3, the consistency
  term equals int eps(p):eps(q) by independent quadrature, the stiffness
  kernel is the 6 rigid motions, and B_K is exact on polynomials.
* Patch test (solenoidal u in [P_k]^3 reproduced) and BDDC-PCG = direct
  solve with lambda_min = 1 on an OCTA mesh.
"""
import os

import numpy as np
import pytest

from synth.mesh import octa_mesh, box_partition
from oracle.poly import dim3, mono3, dmono3
from oracle.vem import Topology, DofMap, System, build_element, total_dofs
from oracle.bddc import BDDC

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    rows = []
    for line in open(os.path.join(HERE, "golden", "paper_dof_counts_octa.txt")):
        if line.startswith("#") or not line.strip():
            continue
        m, k, nd = line.split()[:3]
        rows.append((int(m), int(k), int(nd)))
    return rows


@pytest.mark.parametrize("m,k,ndofs", _golden())
def test_dof_counts_match_paper_tables(m, k, ndofs):
    topo = Topology(octa_mesh(m))
    assert topo.nE == 9 * m ** 3
    assert total_dofs(topo.nV, topo.nEd, topo.nF, topo.nE, k) == ndofs


def _face_vec(xyz, loop):
    P = xyz[list(loop)]
    return 0.5 * sum(np.cross(P[i], P[(i + 1) % len(P)]) for i in range(len(P)))


def test_mesh_is_a_conforming_partition_of_the_cube():
    mesh = octa_mesh(2)
    xyz, fp, fv = mesh["xyz"], mesh["face_ptr"], mesh["face_vtx"]
    ep, ef = mesh["elem_ptr"], mesh["elem_face"]
    nF = len(fp) - 1
    loops = [fv[fp[f]:fp[f + 1]] for f in range(nF)]
    # planar faces
    for lp in loops:
        P = xyz[lp]
        nrm = _face_vec(xyz, lp)
        nrm /= np.linalg.norm(nrm)
        assert np.abs((P - P.mean(0)) @ nrm).max() < 1e-14
    uses = np.zeros(nF, dtype=int)
    sgn = np.zeros(nF, dtype=int)
    vol = 0.0
    for e in range(len(ep) - 1):
        closure = np.zeros(3)
        for s in ef[ep[e]:ep[e + 1]]:
            f = abs(int(s)) - 1
            a = np.sign(s) * _face_vec(xyz, loops[f])
            closure += a
            # divergence theorem with x: |K| = (1/3) sum_f x_f . n_f |f|
            vol += xyz[loops[f]].mean(0) @ a / 3.0
            uses[f] += 1
            sgn[f] += int(np.sign(s))
        assert np.abs(closure).max() < 1e-14
    assert abs(vol - 1.0) < 1e-12
    assert uses.max() == 2
    assert np.all(sgn[uses == 2] == 0)
    # boundary faces lie on the cube's faces
    for f in np.nonzero(uses == 1)[0]:
        P = xyz[loops[f]]
        assert any(np.all(np.abs(P[:, c] - v) < 1e-15) for c in range(3) for v in (0.0, 1.0))


@pytest.fixture(scope="module", params=[(2, 0), (2, 8), (3, 0), (3, 8)],
            ids=["k2-cube", "k2-octa", "k3-cube", "k3-octa"])
def element(request):
    k, e = request.param
    topo = Topology(octa_mesh(1))
    return build_element(topo, DofMap(topo, k), e, 1.0)


def test_element_shapes(element):
    nf = 8 if element.e == 8 else 7
    assert len(element.faces) == nf


def test_projectors_reproduce_polynomials(element):
    I = np.eye(element.D.shape[1])
    tol = {2: 1e-12, 3: 1e-10}[element.k]
    assert np.abs(element.PiN @ element.D - I).max() < tol
    assert np.abs(element.Pi0 @ element.D - I).max() < tol


def test_consistency_on_polynomials(element):
    el = element
    k, hK = el.k, el.hK
    Nk = dim3(k)
    xi = (el.vq_pts - el.xK) / hK
    dm = [dmono3(k, xi, j) / hK for j in range(3)]
    G = np.zeros((len(xi), 3 * Nk, 3, 3))
    for c in range(3):
        for j in range(3):
            G[:, c * Nk:(c + 1) * Nk, c, j] = dm[j]
    E = 0.5 * (G + np.swapaxes(G, 2, 3))
    rhs = np.einsum("p,paij,pbij->ab", el.vq_w, E, E)
    lhs = el.D.T @ el.A @ el.D
    assert np.abs(lhs - rhs).max() < 1e-10 * max(1.0, np.abs(rhs).max())


def test_stiffness_kernel_is_rigid_motions(element):
    ev = np.linalg.eigvalsh(0.5 * (element.A + element.A.T))
    assert np.sum(np.abs(ev) < 1e-9 * ev[-1]) == 6
    assert ev[0] > -1e-9 * ev[-1]


def test_divergence_rows_exact(element):
    k, hK = element.k, element.hK
    Nk = dim3(k)
    M = mono3(k - 1, element.xi)
    ref = np.zeros((dim3(k - 1), 3 * Nk))
    for c in range(3):
        ref[:, c * Nk:(c + 1) * Nk] = (M * element.vq_w[:, None]).T @ (dmono3(k, element.xi, c) / hK)
    got = element.B @ element.D
    assert np.abs(got - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("m,k", [(1, 2), (1, 3)])
def test_patch_test(m, k):
    """Solenoidal u in [P_k]^3, p in P_1 with Dirichlet data of u: the
    discrete solution is the interpolant (convergence theorem, s = k)."""
    mesh = octa_mesh(m)
    b = np.array([1.0, 2.0, -3.0])
    u = lambda x: np.stack([x[:, 1] ** k + x[:, 2], x[:, 2] ** k + x[:, 0], x[:, 0] ** k + x[:, 1]], 1)
    lap = lambda x: np.stack([k * (k - 1) * x[:, 1] ** (k - 2), k * (k - 1) * x[:, 2] ** (k - 2),
                              k * (k - 1) * x[:, 0] ** (k - 2)], 1)
    f = lambda x: -0.5 * lap(x) - b
    nE = len(mesh["elem_ptr"]) - 1
    S = System(mesh, k, np.ones(nE), f=f)
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
    assert np.abs(uh - uI).max() < 1e-10 * np.abs(uI).max()
    assert np.abs(ph - pex).max() < 1e-8 * np.abs(pex).max()
    assert np.abs(S.B @ uh).max() < 1e-11


def test_bddc_pcg_matches_direct_solve():
    """octa_mesh(2) (72 elements), one 2x2x2 block of cubes and its
    octahedron per subdomain: PCG with deluxe scaling reproduces the direct
    solve and lambda_min(M^{-1} S^) = 1."""
    from synth.fields import manufactured_f
    mesh = octa_mesh(2)
    nE = len(mesh["elem_ptr"]) - 1
    part = box_partition(mesh, (2, 2, 2))
    for p in range(8):
        assert np.sum(part == p) == 9
    S = System(mesh, 2, np.ones(nE), f=lambda x: manufactured_f(x, 1.0), load_deg=6)
    u, p = S.solve_direct()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    res = BDDC(S, part, scaling="deluxe").pcg(F, rtol=1e-10)
    assert res["lam_min"] > 1.0 - 1e-8
    uf = u[S.dm.free]
    assert np.linalg.norm(res["x"][:len(uf)] - uf) < 1e-8 * np.linalg.norm(uf)

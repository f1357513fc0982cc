"""Pins of the CVT mesh family (centroidal Voronoi tessellations of the
unit cube, seeded, Lloyd-relaxed) and of the oracle's VEM on Voronoi cells.

* The mesh is a valid conforming polyhedral partition of the cube: closed
  elements, planar convex faces, volumes summing to 1, every interior face
  shared by two elements with opposite orientation.
* The paper's CVT meshes are not available, so their DOF counts cannot be
  matched exactly.  A CVT of the same number of cells has the same counts
  per cell up to boundary and relaxation effects: the 125-cell mesh of the
  degree test (8,945 / 19,256 / 33,487 DOFs at k = 2, 3, 4, which fix its
  vertex, edge and face counts at 643, 1,282 and 765) is matched within 4%.
* On a Voronoi cell (up to 30 vertices, 17 faces, faces of up to 8
  vertices): the projectors reproduce [P_k]^3, the stiffness kernel is the
  6 rigid motions, B_K is exact; the patch test and BDDC-PCG = direct solve
  with lambda_min = 1 on a small CVT mesh.
"""
import functools

import numpy as np
import pytest

from synth.mesh import cvt_mesh
from oracle.poly import dim3, mono3, dmono3
from oracle.vem import Topology, DofMap, System, build_element, total_dofs
from oracle.bddc import BDDC


@functools.lru_cache(maxsize=None)
def _mesh(n, seed, iters):
    return cvt_mesh(n, seed=seed, iters=iters)


def _face_vec(xyz, loop):
    P = xyz[list(loop)]
    return 0.5 * sum(np.cross(P[i], P[(i + 1) % len(P)]) for i in range(len(P)))


def test_mesh_is_a_conforming_partition_of_the_cube():
    mesh = _mesh(64, 3, 20)
    xyz, fp, fv = mesh["xyz"], mesh["face_ptr"], mesh["face_vtx"]
    ep, ef = mesh["elem_ptr"], mesh["elem_face"]
    nF = len(fp) - 1
    loops = [fv[fp[f]:fp[f + 1]] for f in range(nF)]
    for lp in loops:
        P = xyz[lp]
        n = _face_vec(xyz, lp)
        n /= np.linalg.norm(n)
        assert np.abs((P - P.mean(0)) @ n).max() < 1e-8
    uses = np.zeros(nF, dtype=int)
    sgn = np.zeros(nF, dtype=int)
    vol = 0.0
    for e in range(len(ep) - 1):
        closure = np.zeros(3)
        for s in ef[ep[e]:ep[e + 1]]:
            f = abs(int(s)) - 1
            a = np.sign(s) * _face_vec(xyz, loops[f])
            closure += a
            vol += xyz[loops[f]].mean(0) @ a / 3.0
            uses[f] += 1
            sgn[f] += int(np.sign(s))
        assert np.abs(closure).max() < 1e-9
    assert abs(vol - 1.0) < 1e-9
    assert uses.max() == 2 and np.all(sgn[uses == 2] == 0)


@pytest.mark.parametrize("k,ndofs", [(2, 8945), (3, 19256), (4, 33487)])
def test_counts_close_to_the_paper_cvt_mesh(k, ndofs):
    topo = Topology(_mesh(125, 1, 30))
    assert topo.nE == 125
    got = total_dofs(topo.nV, topo.nEd, topo.nF, topo.nE, k)
    assert abs(got - ndofs) <= 0.04 * ndofs


@pytest.fixture(scope="module", params=[2, 3], ids=["k2", "k3"])
def element(request):
    mesh = _mesh(27, 5, 20)
    topo = Topology(mesh)
    # the cell with the most vertices
    e = int(np.argmax([len(v) for v in topo.elem_vertices]))
    return build_element(topo, DofMap(topo, request.param), e, 1.0)


def test_voronoi_cell_projectors_kernel_and_divergence(element):
    el = element
    assert len(el.verts) >= 14
    I = np.eye(el.D.shape[1])
    assert np.abs(el.PiN @ el.D - I).max() < 1e-8
    assert np.abs(el.Pi0 @ el.D - I).max() < 1e-8
    ev = np.linalg.eigvalsh(0.5 * (el.A + el.A.T))
    assert np.sum(np.abs(ev) < 1e-9 * ev[-1]) == 6 and ev[0] > -1e-9 * ev[-1]
    k, hK = el.k, el.hK
    M = mono3(k - 1, el.xi)
    ref = np.zeros((dim3(k - 1), 3 * dim3(k)))
    for c in range(3):
        ref[:, c * dim3(k):(c + 1) * dim3(k)] = (M * el.vq_w[:, None]).T @ (dmono3(k, el.xi, c) / hK)
    assert np.abs(el.B @ el.D - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())


def test_patch_test_on_cvt():
    k = 2
    mesh = _mesh(27, 5, 20)
    b = np.array([1.0, 2.0, -3.0])
    u = lambda x: np.stack([x[:, 1] ** 2 + x[:, 2], x[:, 2] ** 2 + x[:, 0], x[:, 0] ** 2 + x[:, 1]], 1)
    f = lambda x: -np.ones((len(x), 3)) - b
    nE = len(mesh["elem_ptr"]) - 1
    S = System(mesh, k, np.ones(nE), f=f)
    uI = np.zeros(S.dm.nvel)
    for e, el in S.elements.items():
        uI[el.dofs] = el.poly_dofs(u, lambda x: np.zeros(len(x)))
    uh, ph = S.solve_direct(u_bnd=uI)
    assert np.abs(uh - uI).max() < 1e-8 * np.abs(uI).max()
    assert np.abs(S.B @ uh).max() < 1e-10


def test_bddc_pcg_on_cvt():
    """27-cell CVT, two subdomains split by the seed's x coordinate: PCG
    reproduces the direct solve and lambda_min = 1."""
    from synth.fields import manufactured_f
    mesh = _mesh(27, 5, 20)
    nE = len(mesh["elem_ptr"]) - 1
    part = (mesh["seeds"][:, 0] > 0.5).astype(np.int32)
    S = System(mesh, 2, np.ones(nE), f=lambda x: manufactured_f(x, 1.0), load_deg=6)
    u, p = S.solve_direct()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    res = BDDC(S, part, scaling="deluxe").pcg(F, rtol=1e-10)
    assert res["lam_min"] > 1.0 - 1e-8
    uf = u[S.dm.free]
    assert np.linalg.norm(res["x"][:len(uf)] - uf) < 1e-8 * np.linalg.norm(uf)

"""GPU parity, through the C-ABI, of extensions of the BDDC-PCG path
against the CPU oracle:

* deluxe scaling on macro edges (bddc_setup scaling 2): D_E^(k) =
  (sum_j S_E^(j))^{-1} S_E^(k) over the subdomains sharing an edge (the Sec.
  6 formula over card(E) >= 3 subdomains), on a split-hex mesh, an uneven
  greedy partition, a viscosity contrast of 1e4 and an OCTA mesh;
* the OCTA mesh family (octahedra embedded in 2x2x2 blocks of cubes, cubes
  with one truncated corner, pentagonal faces): element matrices at k = 2,
  3, 4, global CSR and load, BDDC-PCG, and the paper's 15,552-element OCTA
  mesh by properties;
* the CVT mesh family (Lloyd-relaxed Voronoi cells: up to about 30
  vertices, faces of up to 9 vertices, some of them thin): element
  matrices, load and BDDC-PCG;
* the reduced scheme (vem_assemble_reduced: D5 eliminated with value 0,
  element-constant pressure): element matrices, CSR and load against the
  oracle's reduced System, BDDC-PCG against the oracle's BDDC on it, and
  the velocity against the full scheme's direct solve.

Tolerances as in the other parity tests: element matrices and assembly to
rounding; PCG by the shared rule of oracle_cache.check_pcg_parity
(iterations within +-1 of the oracle's, or of its own range under
rounding-level perturbation; lambda_max within 1e-6; at equal iteration
counts the velocity and the whole zero-mean solution within 1e-10, and at
rtol 1e-11 within 1e-10 wherever the oracle cannot reproduce its own
iterate to 1e-11).
"""
import numpy as np
import pytest

from synth import make_config
from oracle.vem import Topology, DofMap, System, build_element
from oracle_cache import oracle_system, oracle_bddc, check_pcg_parity

pytestmark = pytest.mark.gpu

SCALING = {"multiplicity": 0, "deluxe": 1, "deluxe_edges": 2}


def _deep(bd, rhs):
    """The same GPU solve to a tighter rtol (for the converged comparison)."""
    def run(rtol):
        import torch
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=rtol, maxit=2000)
        assert res["status"] == 0
        return res, u.cpu().numpy()
    return run


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2304_09770_gb300 as p
    p.lib()
    return p


def _setup(pkg, name):
    cfg, S = oracle_system(name)
    k = cfg["k"]
    deg = k + 9 if cfg["spec"]["load"] == "manufactured" else 2 * k + 2
    g = pkg.VemSystem(cfg["mesh"], k, cfg["nu"])
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    return cfg, g, rhs, S, F


@pytest.mark.parametrize("name,tol", [("octa2_k2", 1e-12), ("octa2_k3", 1e-11), ("octa2_k4", 1e-9)])
def test_octa_element_matrices_match_oracle(pkg, name, tol):
    cfg = make_config(name)
    g = pkg.VemSystem(cfg["mesh"], cfg["k"], cfg["nu"])
    topo = Topology(cfg["mesh"])
    dm = DofMap(topo, cfg["k"])
    # truncated cubes, then octahedra (one DOF count per call)
    for elems in ([0, 5, 21, 42, 63], [64, 67, topo.nE - 1]):
        A, B, D = g.element_matrices(elems)
        for i, e in enumerate(elems):
            el = build_element(topo, dm, e, cfg["nu"][e])
            assert np.array_equal(D[i], el.dofs)
            assert np.abs(A[i] - el.A).max() <= tol * np.abs(el.A).max()
            assert np.abs(B[i] - el.B).max() <= tol * np.abs(el.B).max()


def test_octa_global_matrix_and_load_match_oracle(pkg):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, "octa2_k2")
    assert np.array_equal(g.free_dofs(), S.dm.free)
    Kg = g.csr().toarray()
    Ko = S.free_matrix().toarray()
    assert np.abs(Kg - Ko).max() <= 1e-12 * np.abs(Ko).max()
    got = rhs.cpu().numpy()
    assert np.abs(got - F).max() <= 1e-12 * np.abs(F).max()
    x = torch.randn(g.n, dtype=torch.float64, device="cuda")
    y = g.apply(x).cpu().numpy()
    yo = Ko @ x.cpu().numpy()
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("name,tol", [("cvt64_k2", 1e-12), ("cvt27_k3", 1e-11)])
def test_cvt_element_matrices_and_load_match_oracle(pkg, name, tol):
    cfg, g, rhs, S, F = _setup(pkg, name)
    topo = S.topo
    # Voronoi cells differ in their DOF counts: one element per call
    for e in range(0, topo.nE, max(1, topo.nE // 8)):
        A, B, D = g.element_matrices([e])
        el = S.elements[e]
        assert np.array_equal(D[0], el.dofs)
        assert np.abs(A[0] - el.A).max() <= tol * np.abs(el.A).max()
        assert np.abs(B[0] - el.B).max() <= tol * np.abs(el.B).max()
    assert np.abs(rhs.cpu().numpy() - F).max() <= tol * np.abs(F).max()


CASES = [("tri6_k2", "deluxe_edges"), ("tri6_greedy", "deluxe_edges"), ("sinker8", "deluxe_edges"),
         ("octa2_k2", "deluxe"), ("octa2_k2", "deluxe_edges"), ("octa2_k3", "deluxe"),
         ("octa2_sinker", "deluxe"), ("octa2_sinker", "deluxe_edges"),
         ("cvt64_k2", "deluxe"), ("cvt64_k2", "deluxe_edges"), ("cvt27_k3", "deluxe")]


@pytest.mark.parametrize("name,scaling", CASES)
def test_pcg_matches_oracle(pkg, name, scaling):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, name)
    bd = pkg.Bddc(g, cfg["part"], constraints=15, scaling=SCALING[scaling])
    if scaling == "deluxe_edges":
        assert bd.info("n_deluxe_edges") > 0
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=300)
    assert res["status"] == 0
    assert res["lam_min"] > 1.0 - 1e-8
    _, _, ob, _ = oracle_bddc(name, scaling=scaling)
    check_pcg_parity(S, ob, F, res, u.cpu().numpy(), label=f"{name}-{scaling}", deep=_deep(bd, rhs))


@pytest.mark.parametrize("name,scaling", [("tri6_k2", "deluxe_edges"), ("tri6_greedy", "deluxe_edges"),
                                          ("octa2_k2", "deluxe_edges")])
def test_preconditioner_matches_oracle(pkg, name, scaling):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, name)
    bd = pkg.Bddc(g, cfg["part"], scaling=SCALING[scaling])
    _, _, ob, _ = oracle_bddc(name, scaling=scaling)
    r = F - ob.K @ ob.initial_guess(F)
    zo = ob.apply(r)
    z = bd.apply(torch.tensor(r, device="cuda")).cpu().numpy()
    nvf = len(S.dm.free)
    assert np.abs(z[:nvf] - zo[:nvf]).max() <= 1e-11 * np.abs(zo[:nvf]).max()
    assert np.abs(z[nvf:] - zo[nvf:]).max() <= 1e-10 * np.abs(zo[nvf:]).max()


def test_edge_deluxe_lowers_kappa_at_contrast(pkg):
    """8^3 cubes with 8 sinkers (contrast 1e4): deluxe weights on the edges
    follow the coefficient jump; kappa falls well below face-only deluxe
    (the oracle gives 133.6 -> 48.4)."""
    import torch
    cfg, g, rhs, S, F = _setup(pkg, "sinker8")
    out = {}
    for sc in ("deluxe", "deluxe_edges"):
        bd = pkg.Bddc(g, cfg["part"], scaling=SCALING[sc])
        u = torch.zeros_like(rhs)
        out[sc] = bd.solve(rhs, u, rtol=1e-8, maxit=300)
    assert out["deluxe_edges"]["kappa"] < 0.5 * out["deluxe"]["kappa"]
    assert out["deluxe_edges"]["iters"] < out["deluxe"]["iters"]


def test_invalid_scaling_is_rejected(pkg):
    cfg = make_config("cube4_k2")
    g = pkg.VemSystem(cfg["mesh"], cfg["k"], cfg["nu"])
    with pytest.raises(pkg.VemError) as e:
        pkg.Bddc(g, cfg["part"], scaling=3)
    assert e.value.status == -1


def test_octa_full_size_properties(pkg):
    """The paper's OCTA mesh of its strong-scaling and sinker tests: 15,552
    elements, 549,939 DOFs at k = 2, 64 subdomains.  Converges, lambda_min
    >= 1, the saddle-system residual is at the CG tolerance and the discrete
    velocity is divergence-free elementwise."""
    import torch
    cfg = make_config("octa12_k2")
    deg = 11
    g = pkg.VemSystem(cfg["mesh"], 2, cfg["nu"])
    assert g.n_vel + g.n_press == 549939
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    bd = pkg.Bddc(g, cfg["part"])
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=500)
    assert res["status"] == 0
    assert res["lam_min"] > 1.0 - 1e-8
    r = rhs - g.apply(u)
    assert torch.linalg.norm(r).item() <= 1e-7 * torch.linalg.norm(rhs).item()
    assert torch.abs(r[g.n_vel_free:]).max().item() <= 1e-7 * torch.abs(rhs).max().item()


def _setup_reduced(pkg, name):
    cfg, S = oracle_system(name, reduced=True)
    k = cfg["k"]
    deg = k + 9
    g = pkg.VemSystem(cfg["mesh"], k, cfg["nu"], reduced=True)
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    return cfg, g, rhs, S, F


@pytest.mark.parametrize("name", ["tri4_k2", "octa2_k3"])
def test_reduced_system_matches_oracle(pkg, name):
    cfg, g, rhs, S, F = _setup_reduced(pkg, name)
    assert g.info("reduced") == 1.0
    assert g.n_press == S.topo.nE and np.array_equal(g.free_dofs(), S.dm.free)
    elems = [0, 5, 21]
    A, B, D = g.element_matrices(elems)
    for i, e in enumerate(elems):
        el = S.elements[e]
        assert np.abs(A[i] - el.A).max() <= 1e-11 * np.abs(el.A).max()
        assert B.shape[1] == 1 and np.abs(B[i, 0] - el.B[0]).max() <= 1e-11 * np.abs(el.B[0]).max()
    Kg = g.csr().toarray()
    Ko = S.free_matrix().toarray()
    assert np.abs(Kg - Ko).max() <= 1e-12 * np.abs(Ko).max()
    assert np.abs(rhs.cpu().numpy() - F).max() <= 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("name,scaling", [("tri4_k2", "deluxe"), ("octa2_k3", "deluxe_edges"),
                                          ("tri6_k2", "deluxe")])
def test_reduced_pcg_matches_oracle(pkg, name, scaling):
    import torch
    cfg, g, rhs, S, F = _setup_reduced(pkg, name)
    bd = pkg.Bddc(g, cfg["part"], scaling=SCALING[scaling])
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=300)
    assert res["status"] == 0 and res["lam_min"] > 1.0 - 1e-8
    _, _, ob, _ = oracle_bddc(name, scaling=scaling, reduced=True)
    check_pcg_parity(S, ob, F, res, u.cpu().numpy(), label=f"reduced-{name}-{scaling}", deep=_deep(bd, rhs))
    nvf = len(S.dm.free)
    x = u.cpu().numpy()
    # the same velocity as the full scheme (its direct solve), within the CG tolerance
    _, full = oracle_system(name)
    ud, _ = full.solve_direct()
    ur = np.zeros(S.dm.nvel)
    ur[S.dm.free] = x[:nvf]
    assert np.linalg.norm(ur - ud) <= 1e-6 * np.linalg.norm(ud)


def test_reduced_full_size_properties(pkg):
    """The reduced scheme on the 32^3 benchmark mesh: 6 fewer unknowns per
    element, converges with lambda_min >= 1, the residual of the reduced
    saddle system is at the CG tolerance, and the velocity equals the full
    scheme's (both solved by BDDC-PCG to rtol 1e-10)."""
    import torch
    cfg = make_config("tri32_k2")
    deg = 6
    out = {}
    for reduced in (False, True):
        g = pkg.VemSystem(cfg["mesh"], 2, cfg["nu"], reduced=reduced)
        rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
        bd = pkg.Bddc(g, cfg["part"])
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=1e-10, maxit=500)
        assert res["status"] == 0 and res["lam_min"] > 1.0 - 1e-8
        r = rhs - g.apply(u)
        assert torch.linalg.norm(r).item() <= 1e-9 * torch.linalg.norm(rhs).item()
        uv = np.zeros(g.n_vel)
        uv[g.free_dofs()] = u[:g.n_vel_free].cpu().numpy()
        out[reduced] = (g.n, uv)
        del bd, g
    nE = 32 ** 3
    assert out[False][0] - out[True][0] == 6 * nE
    a, b = out[False][1], out[True][1]
    assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(a)

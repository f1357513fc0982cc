"""Pins of the oracle's BDDC-PCG against what the paper's theory fixes:
lambda_min(M^{-1} S^) = 1 (Theorem on the benign space), one iteration when
every interface DOF is primal, a single subdomain reduces to the direct solve,
symmetry of M^{-1}, D_F^(i) + D_F^(j) = I, E_D a projection, and PCG = direct
solve within the CG tolerance."""
import numpy as np
import pytest

from synth import make_config, cube_mesh, box_partition
from oracle.vem import System
from oracle.bddc import BDDC


@pytest.fixture(scope="module", params=["cube4_k2", "tri4_k2"])
def system(request):
    cfg = make_config(request.param)
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"])
    u, p = S.solve_direct()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    return cfg, S, u, p, F


def _errs(S, x, u, p):
    nvf = len(S.dm.free)
    uf = u[S.dm.free]
    pp = x[nvf:] - (S.wmean @ x[nvf:]) / S.wmean.sum()
    return (np.linalg.norm(x[:nvf] - uf) / np.linalg.norm(uf),
            np.linalg.norm(pp - p) / np.linalg.norm(p))


@pytest.mark.parametrize("scaling", ["deluxe", "multiplicity"])
def test_pcg_matches_direct_and_lambda_min(system, scaling):
    cfg, S, u, p, F = system
    bd = BDDC(S, cfg["part"], scaling=scaling)
    res = bd.pcg(F, rtol=1e-10)
    eu, ep = _errs(S, res["x"], u, p)
    assert eu < 1e-8 and ep < 1e-6
    assert res["lam_min"] > 1.0 - 1e-8
    assert res["kappa"] < 20.0


def test_all_primal_is_exact(system):
    cfg, S, u, p, F = system
    bd = BDDC(S, cfg["part"], constraints="all", scaling="multiplicity")
    res = bd.pcg(F, rtol=1e-10)
    assert res["iters"] == 1
    assert abs(res["lam_min"] - 1.0) < 1e-8 and abs(res["lam_max"] - 1.0) < 1e-8


def test_single_subdomain_is_direct_solve():
    cfg = make_config("tri4_k2")
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"])
    u, p = S.solve_direct()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    bd = BDDC(S, np.zeros(S.topo.nE, dtype=np.int32))
    res = bd.pcg(F)
    assert res["iters"] == 0
    eu, ep = _errs(S, res["x"], u, p)
    assert eu < 1e-12 and ep < 1e-10


def test_preconditioner_symmetric_and_deluxe_partition_of_unity(system):
    cfg, S, u, p, F = system
    bd = BDDC(S, cfg["part"], scaling="deluxe")
    rng = np.random.default_rng(5)
    rs = []
    for _ in range(2):
        # residuals of harmonic fields: interior rows zero
        x = np.zeros(bd.nvf + bd.npr)
        x[:bd.nvf] = rng.standard_normal(bd.nvf) * (bd.mult >= 2)
        for sub in bd.subs:
            nI = sub["nI"]
            v = sub["T"].T @ x[sub["vel"]]
            v[:nI] = 0
            zI, zp = bd._dirichlet(sub, -(sub["At"][:nI] @ v), -(sub["Bt"] @ v))
            x[sub["vel"][sub["interior"]]] = zI
            x[bd.nvf + sub["prs"]] = zp
        rs.append(bd.K @ x)
    z0, z1 = bd.apply(rs[0]), bd.apply(rs[1])
    a, b = rs[1] @ z0, rs[0] @ z1
    assert abs(a - b) < 1e-9 * max(abs(a), abs(b))
    assert len(bd.DF) > 0
    for gi, D in bd.DF.items():
        i, j = bd.macro[gi]["share"]
        assert np.abs(D[i] + D[j] - np.eye(len(D[i]))).max() < 1e-10


def test_averaging_is_a_projection(system):
    """E_D = R~ R~_D^T: averaging an already continuous field returns it."""
    cfg, S, u, p, F = system
    bd = BDDC(S, cfg["part"], scaling="deluxe")
    rng = np.random.default_rng(9)
    for gi, G in enumerate(bd.macro):
        if gi not in bd.DF:
            continue
        w = rng.standard_normal(G["ndual"])
        i, j = G["share"]
        avg = bd._scale(gi, i, w) + bd._scale(gi, j, w)
        assert np.abs(avg - w).max() < 1e-10
        wi, wj = rng.standard_normal(G["ndual"]), rng.standard_normal(G["ndual"])
        once = bd._scale(gi, i, wi) + bd._scale(gi, j, wj)
        twice = bd._scale(gi, i, once) + bd._scale(gi, j, once)
        assert np.abs(twice - once).max() < 1e-10


def test_flux_primal_gives_benign_dual_space(system):
    """Every dual coordinate of a macro face has zero normal flux (Assumption 1)."""
    cfg, S, u, p, F = system
    bd = BDDC(S, cfg["part"])
    for G in bd.macro:
        if G["kind"] != "face" or G["ndual"] == 0:
            continue
        C = G["C"]
        Qd = G["T"][:, :G["ndual"]]
        assert np.abs(C @ Qd).max() < 1e-10


def test_adaptive_eigenvalues_and_monotonicity():
    """Adaptive coarse space (Sec. 6) on the 4^3 perturbed mesh: since the
    Neumann Schur complement onto a face is below the principal minor of
    the Dirichlet one (S~ <= S, more freedom lowers the energy) and parallel
    sums are monotone, every eigenvalue of (S~_i : S~_j, S_i : S_j) lies in
    (0, 1]; lowering theta (raising the cut 1/theta) adds functionals and
    does not raise kappa; lambda_min stays 1 (Theorem on the benign space)."""
    cfg = make_config("tri4_k2")
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=6)
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    added, kappas = [], []
    for theta in (10.0, 2.0, 1.1):
        b = BDDC(S, cfg["part"], adaptive=theta)
        eigs = np.concatenate(list(b.adapt_eigs.values()))
        assert eigs.min() > 0.0 and eigs.max() <= 1.0 + 1e-10
        r = b.pcg(F, rtol=1e-8)
        assert r["lam_min"] > 1.0 - 1e-8
        added.append(b.n_adaptive)
        kappas.append(r["lam_max"] / r["lam_min"])
        assert b.n_adaptive == int((eigs < 1.0 / theta).sum())
    assert added[0] <= added[1] <= added[2] and added[2] > added[0]
    assert kappas[0] >= kappas[1] - 1e-8 >= kappas[2] - 2e-8

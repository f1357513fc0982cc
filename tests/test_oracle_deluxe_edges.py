"""Pins of the oracle's deluxe scaling extended to macro edges (the deluxe
formula of Sec. 6, D_G^(k) = (sum_{j in N_G} S_G^(j))^{-1} S_G^(k), taken
over the card(N_E) >= 3 subdomains of an edge instead of 1/card, Eq.
pseudoinv).

What fixes it independently of the oracle's own bookkeeping:
* S_G^(k) equals V^T S^(k) V, with S^(k) the dense Schur complement of the
  subdomain's matrix in the original DOF basis (interior velocity and the
  zero-mean pressure eliminated, Eq. uipi) and V the dual basis vectors of
  G written out in global DOFs: this checks the blocks are taken on the
  right coordinates of the right entity.
* sum_k D_G^(k) = I and the averaging is a projection (Sec. 4.3).
* M^{-1} stays symmetric and lambda_min(M^{-1} S^) = 1: the edge dual
  coordinates carry no face flux, so the averaging still preserves the
  subdomain normal fluxes (Theorem on the benign space); PCG reproduces the
  direct solve.
* At a viscosity contrast (8 sinkers) the edge deluxe weights follow the
  coefficient jump that counting ignores: kappa drops well below the
  face-only deluxe value.
"""
import numpy as np
import pytest

from synth import make_config
from oracle.vem import System
from oracle.bddc import BDDC


@pytest.fixture(scope="module", params=["cube4_k2", "tri4_k2"])
def case(request):
    cfg = make_config(request.param)
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"])
    u, p = S.solve_direct()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    bd = BDDC(S, cfg["part"], scaling="deluxe_edges")
    return cfg, S, u, p, F, bd


def _dense_schur(S, bd, i):
    """Schur complement of subdomain i onto its interface velocity DOFs, in
    the original DOF basis, by dense elimination of the interior velocity
    and of the pressure with a zero (weighted) mean."""
    vel, prs = bd.vel[i], bd.prs[i]
    idx = np.concatenate([vel, bd.nvf + prs])
    K = S.local_matrix(np.nonzero(bd.part == i)[0])[idx][:, idx].toarray()
    nv, npl = len(vel), len(prs)
    A, B = K[:nv, :nv], K[nv:, :nv]
    gam = np.nonzero(bd.mult[vel] >= 2)[0]
    inn = np.nonzero(bd.mult[vel] < 2)[0]
    w = S.wmean[prs]
    nI = len(inn)
    M = np.zeros((nI + npl + 1, nI + npl + 1))
    M[:nI, :nI] = A[np.ix_(inn, inn)]
    M[:nI, nI:nI + npl] = B[:, inn].T
    M[nI:nI + npl, :nI] = B[:, inn]
    M[nI:nI + npl, -1] = w
    M[-1, nI:nI + npl] = w
    C = np.zeros((nI + npl + 1, len(gam)))
    C[:nI] = A[np.ix_(inn, gam)]
    C[nI:nI + npl] = B[:, gam]
    X = np.linalg.solve(M, C)
    Sg = A[np.ix_(gam, gam)] - C.T @ X
    return vel[gam], 0.5 * (Sg + Sg.T)


def test_blocks_are_principal_minors_of_the_schur_complement(case):
    cfg, S, u, p, F, bd = case
    kinds = {bd.macro[gi]["kind"] for gi in bd.DF}
    assert kinds == {"face", "edge"}
    for i in range(bd.N):
        gdofs, Sg = _dense_schur(S, bd, i)
        pos = {int(g): a for a, g in enumerate(gdofs)}
        for gi, blocks in bd.SF.items():
            if i not in blocks:
                continue
            G = bd.macro[gi]
            V = np.zeros((len(gdofs), G["ndual"]))
            for a, g in enumerate(G["dofs"]):
                V[pos[int(g)]] = G["T"][a, :G["ndual"]]
            ref = V.T @ Sg @ V
            assert np.abs(blocks[i] - ref).max() < 1e-9 * np.abs(ref).max()


def test_partition_of_unity_and_projection(case):
    cfg, S, u, p, F, bd = case
    rng = np.random.default_rng(3)
    n_edges = 0
    for gi, D in bd.DF.items():
        G = bd.macro[gi]
        share = G["share"]
        assert np.abs(sum(D[s] for s in share) - np.eye(G["ndual"])).max() < 1e-10
        if G["kind"] != "edge":
            continue
        n_edges += 1
        assert len(share) >= 3
        w = rng.standard_normal(G["ndual"])
        assert np.abs(sum(bd._scale(gi, s, w) for s in share) - w).max() < 1e-10
        once = sum(bd._scale(gi, s, rng.standard_normal(G["ndual"])) for s in share)
        twice = sum(bd._scale(gi, s, once) for s in share)
        assert np.abs(twice - once).max() < 1e-10
    assert n_edges > 0


def test_symmetric_lambda_min_one_and_direct_solve(case):
    cfg, S, u, p, F, bd = case
    rng = np.random.default_rng(11)
    rs = []
    for _ in range(2):
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
    a, b = rs[1] @ bd.apply(rs[0]), rs[0] @ bd.apply(rs[1])
    assert abs(a - b) < 1e-9 * max(abs(a), abs(b))
    res = bd.pcg(F, rtol=1e-10)
    assert res["lam_min"] > 1.0 - 1e-8
    nvf = bd.nvf
    uf = u[S.dm.free]
    pp = res["x"][nvf:] - (S.wmean @ res["x"][nvf:]) / S.wmean.sum()
    assert np.linalg.norm(res["x"][:nvf] - uf) < 1e-8 * np.linalg.norm(uf)
    assert np.linalg.norm(pp - p) < 1e-6 * np.linalg.norm(p)


def test_edge_deluxe_at_viscosity_contrast():
    # 4^3 cubes, 2^3 subdomains, the 8 sinkers of the contrast-1e4 case
    # (nu in [1, 5.1e3] at the element centres)
    cfg = make_config("sinker8", n=4)
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=6)
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    out = {}
    for sc in ("deluxe", "deluxe_edges"):
        r = BDDC(S, cfg["part"], scaling=sc).pcg(F, rtol=1e-8)
        assert r["lam_min"] > 1.0 - 1e-8
        out[sc] = r
    # observed: kappa 438 -> 9.4, 58 -> 19 iterations
    assert out["deluxe_edges"]["kappa"] < 0.5 * out["deluxe"]["kappa"]
    assert out["deluxe_edges"]["iters"] < out["deluxe"]["iters"]

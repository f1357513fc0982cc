"""Pins of the preconditioned interface operator's spectrum, computed
densely and independently of CG.

The interface problem (Eq. globInt) acts on (u_Gamma, p_0): interface
velocity DOFs and one constant pressure per subdomain.  Column j of
M^{-1} S^ is obtained by extending the j-th unit vector harmonically
(subdomain Dirichlet solves, Eq. uipi), applying the full saddle matrix,
applying the preconditioner (Eq. BDDCprec) and reading the interface
coordinates back.  Then:

* exactly one eigenvalue vanishes (the global constant pressure, the null
  space of the bordered problem); every other one is >= 1 and the smallest
  is 1 (Theorem: lambda_min(M^{-1} S^) = 1 on the benign space);
* the Lanczos estimate of lambda_max from the CG coefficients (diagonal
  1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j)
  equals the largest eigenvalue of the dense operator.
"""
import numpy as np
import pytest

from synth import make_config
from oracle.vem import System
from oracle.bddc import BDDC


def _dense_operator(bd):
    G = np.nonzero(bd.mult >= 2)[0]
    nG, N = len(G), bd.N

    def extend(e):
        x = np.zeros(bd.nvf + bd.npr)
        x[G] = e[:nG]
        for i, sub in enumerate(bd.subs):
            nI = sub["nI"]
            v = sub["T"].T @ x[sub["vel"]]
            v[:nI] = 0.0
            zI, zp = bd._dirichlet(sub, -(sub["At"][:nI] @ v), -(sub["Bt"] @ v))
            x[sub["vel"][sub["interior"]]] = zI
            x[bd.nvf + sub["prs"]] = zp + e[nG + i] * sub["ones_p"]
        return x

    def coords(z):
        p0 = [(sub["w"] @ z[bd.nvf + sub["prs"]]) / (sub["w"] @ sub["ones_p"]) for sub in bd.subs]
        return np.concatenate([z[G], p0])

    n = nG + N
    P = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        P[:, j] = coords(bd.apply(bd.K @ extend(e)))
    return P


@pytest.mark.parametrize("name,scaling", [("cube4_k2", "deluxe_edges"), ("cube4_k2", "multiplicity"),
                                          ("tri4_k2", "deluxe")])
def test_spectrum_of_the_preconditioned_operator(name, scaling):
    cfg = make_config(name)
    S = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=6)
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    bd = BDDC(S, cfg["part"], scaling=scaling)
    ev = np.linalg.eigvals(_dense_operator(bd))
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev).max()
    ev = np.sort(ev.real)
    assert abs(ev[0]) < 1e-10 * ev[-1]
    assert ev[1] > 1.0 - 1e-8
    assert abs(ev[1] - 1.0) < 1e-8
    res = bd.pcg(F, rtol=1e-13, maxit=500)
    assert abs(res["lam_max"] - ev[-1]) < 1e-6 * ev[-1]
    assert res["lam_min"] > 1.0 - 1e-8

"""Pins of the oracle's reduced scheme (the Remark after the convergence
theorem): velocity restricted to fields with vanishing element divergence
moments of degree >= 1 (D5 = 0), pressure restricted to element constants.

* The full scheme's discrete velocity is divergence-free, so its D5 DOFs
  vanish: it lies in the reduced space (the premise of the Remark).
* The reduced system gives the same velocity as the full one, and the
  full P_{k-1} pressure is recovered element by element from the D5 rows.
* The unknown count drops by 2 dim(P_{k-1}) - 2 per element.
* BDDC-PCG on the reduced system reproduces its direct solve with
  lambda_min = 1.
"""
import functools

import numpy as np
import pytest

from synth import make_config
from oracle.vem import System, counts
from oracle.bddc import BDDC


@functools.lru_cache(maxsize=None)
def _pair(name, **over):
    cfg = make_config(name, **over)
    deg = 6
    full = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=deg)
    red = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=deg, reduced=True)
    return cfg, full, red


def _zero_mean(S, p, w):
    """p minus the constant pressure c with int_Omega (p - c) = 0 (c enters
    the constant coefficient of every element only)."""
    one = np.zeros_like(p)
    one[0::S.dm.c["press"]] = 1.0
    return p - (w @ p) / (w @ one) * one


@pytest.fixture(scope="module", params=[("tri4_k2", {}), ("tri4_k3", {"n": 2}), ("octa2_k2", {"m": 1})],
                ids=["tri4_k2", "tri2_k3", "octa1_k2"])
def pair(request):
    name, over = request.param
    return _pair(name, **over)


def test_unknown_counts(pair):
    cfg, full, red = pair
    c = counts(cfg["k"])
    nE = full.topo.nE
    assert len(full.dm.free) - len(red.dm.free) == nE * c["d5"]
    assert full.dm.npress - red.dm.npress == nE * (c["press"] - 1)


def test_full_velocity_has_no_d5_part(pair):
    cfg, full, red = pair
    u, p = full.solve_direct()
    d5 = red.dm.fixed & ~full.dm.fixed
    assert d5.sum() == full.topo.nE * counts(cfg["k"])["d5"]
    assert np.abs(u[d5]).max() < 1e-10 * np.abs(u).max()


def test_same_velocity_and_recovered_pressure(pair):
    cfg, full, red = pair
    u, p = full.solve_direct()
    ur, p0 = red.solve_direct()
    assert np.abs(ur - u).max() < 1e-10 * np.abs(u).max()
    pr = red.full_pressure(ur, p0)
    a = _zero_mean(full, p, full.wmean)
    b = _zero_mean(full, pr, full.wmean)
    assert np.abs(a - b).max() < 1e-8 * np.abs(a).max()


def test_bddc_on_the_reduced_system():
    cfg, full, red = _pair("tri4_k2")
    ur, p0 = red.solve_direct()
    F = np.concatenate([red.F[red.dm.free], np.zeros(red.dm.npress)])
    res = BDDC(red, cfg["part"], scaling="deluxe").pcg(F, rtol=1e-10)
    assert res["lam_min"] > 1.0 - 1e-8
    uf = ur[red.dm.free]
    assert np.linalg.norm(res["x"][:len(uf)] - uf) < 1e-8 * np.linalg.norm(uf)

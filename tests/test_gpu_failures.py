"""Failure detection of the C ABI on the GPU, with every failure made on the
host or by a bounded wait that runs out (nothing faults, traps or hangs):

* a non-finite right-hand side stops PCG with VEM_EBREAKDOWN, in the
  graph-captured loop and in the host-driven one;
* a partition whose floating subdomain's primal constraints cannot control
  its rigid body modes (Sec. 5.1: the coarse space must contain them) is
  rejected by bddc_setup with VEM_ESINGULAR before any factorization;
* the bounded mbarrier wait of the tensor-core kernels, on a barrier that
  nothing arrives on, gives up and reports VEM_ETIMEOUT, and the context
  stays usable for a solve afterwards.
"""
import ctypes

import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2304_09770_gb300 as p
    p.lib()
    return p


def _system(pkg, name):
    cfg = make_config(name)
    g = pkg.VemSystem(cfg["mesh"], cfg["k"], cfg["nu"])
    deg = cfg["k"] + 9
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    return cfg, g, rhs


@pytest.mark.parametrize("use_graph", [0, -1])
@pytest.mark.parametrize("where", ["velocity", "pressure"])
def test_nan_right_hand_side_is_a_breakdown(pkg, use_graph, where):
    import torch
    cfg, g, rhs = _system(pkg, "cube4_k2")
    bd = pkg.Bddc(g, cfg["part"], use_graph=use_graph)
    f = rhs.clone()
    # the largest velocity row, or the last pressure row
    idx = int(np.argmax(np.abs(rhs[:g.n_vel_free].cpu().numpy()))) if where == "velocity" else g.n - 1
    f[idx] = float("nan")
    with pytest.raises(pkg.VemError) as e:
        bd.solve(f, torch.zeros_like(f), rtol=1e-8, maxit=50)
    assert e.value.status == -5
    # the handle still solves a finite problem afterwards
    u = torch.zeros_like(rhs)
    assert bd.solve(rhs, u, rtol=1e-8, maxit=50)["status"] == 0


def test_floating_subdomain_without_rigid_mode_control_is_singular(pkg):
    import torch
    # 6^3 cubes in 3 x 3 x 3 subdomains: the centre one touches no Dirichlet
    # boundary.  Face fluxes alone (constraints = 8) cannot control the
    # rotations of a box (their normal fluxes vanish on every face).
    cfg, g, rhs = _system(pkg, "cube6_k2")
    with pytest.raises(pkg.VemError) as e:
        pkg.Bddc(g, cfg["part"], constraints=8)
    assert e.value.status == -4 and "rigid body modes" in str(e.value)
    with pytest.raises(pkg.VemError) as e:
        pkg.Bddc(g, cfg["part"], constraints=0)
    assert e.value.status == -4
    # the default vertex + edge + face + flux set passes the same check
    bd = pkg.Bddc(g, cfg["part"], constraints=15)
    assert bd.solve(rhs, torch.zeros_like(rhs), rtol=1e-8, maxit=100)["status"] == 0


def test_bounded_wait_gives_up_with_etimeout(pkg):
    import torch
    L = pkg.lib()
    L.vem_wait_selftest.argtypes = [ctypes.c_longlong]
    assert L.vem_wait_selftest(1000) == -7
    assert b"gave up" in L.vem_last_error()
    assert L.vem_wait_selftest(-1) == -1
    # the context is still usable
    cfg, g, rhs = _system(pkg, "cube4_k2")
    bd = pkg.Bddc(g, cfg["part"])
    assert bd.solve(rhs, torch.zeros_like(rhs), rtol=1e-8, maxit=50)["status"] == 0

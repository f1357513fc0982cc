"""GPU parity of BDDC-PCG against the CPU oracle, through the C-ABI: the
iteration count within +-1 and, at equal iteration counts, the velocity and
the zero-mean pressure within 1e-10 relative to the oracle's PCG iterate;
the Lanczos estimates, lambda_min >= 1, the preconditioner itself, and
properties at the full benchmark size."""
import numpy as np
import pytest

from synth import make_config
from oracle_cache import oracle_system, oracle_bddc, check_pcg_parity

pytestmark = pytest.mark.gpu

CONS = {"vertex": 1, "edge": 2, "face": 4, "flux": 8}


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2304_09770_gb300 as p
    p.lib()
    return p


def _setup(pkg, name, **overrides):
    cfg, S = oracle_system(name, **overrides)
    k = cfg["k"]
    deg = k + 9 if cfg["spec"]["load"] == "manufactured" else 2 * k + 2
    g = pkg.VemSystem(cfg["mesh"], k, cfg["nu"])
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    return cfg, g, rhs, S, F


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
CASES = [("cube4_k2", "deluxe"), ("tri4_k2", "deluxe"), ("tri6_k2", "deluxe"), ("tri6_k2", "multiplicity"),
         ("tri4_k3", "deluxe"), ("cube6_k2", "deluxe"), ("sinker8", "deluxe"), ("tri6_greedy", "deluxe")]


@pytest.mark.parametrize("name,scaling", CASES)
def test_pcg_matches_oracle(pkg, name, scaling):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, name)
    bd = pkg.Bddc(g, cfg["part"], constraints=15, scaling=SCALING[scaling])
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=300)
    assert res["status"] == 0
    assert res["lam_min"] > 1.0 - 1e-8
    _, _, ob, _ = oracle_bddc(name, scaling=scaling)
    check_pcg_parity(S, ob, F, res, u.cpu().numpy(), label=f"{name}-{scaling}", deep=_deep(bd, rhs))
    # against the direct solve of the saddle system, within the CG tolerance
    x = u.cpu().numpy()
    nvf = len(S.dm.free)
    ud, pd = S.solve_direct(F=S.F)
    assert np.linalg.norm(x[:nvf] - ud[S.dm.free]) <= 1e-6 * np.linalg.norm(ud[S.dm.free])


def test_all_interface_primal_is_one_iteration(pkg):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, "tri4_k2")
    bd = pkg.Bddc(g, cfg["part"], constraints=16, scaling=0)
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-10, maxit=10)
    assert res["status"] == 0 and res["iters"] == 1
    assert abs(res["lam_min"] - 1.0) < 1e-8


@pytest.mark.parametrize("name,scaling", [("tri6_k2", "deluxe")])
def test_preconditioner_matches_oracle(pkg, name, scaling):
    import torch
    cfg, g, rhs, S, F = _setup(pkg, name)
    bd = pkg.Bddc(g, cfg["part"], scaling=SCALING[scaling])
    _, _, ob, _ = oracle_bddc(name, scaling=scaling)
    x0 = ob.initial_guess(F)
    r = F - ob.K @ x0
    zo = ob.apply(r)
    z = bd.apply(torch.tensor(r, device="cuda")).cpu().numpy()
    nvf = len(S.dm.free)
    assert np.abs(z[:nvf] - zo[:nvf]).max() <= 1e-11 * np.abs(zo[:nvf]).max()
    assert np.abs(z[nvf:] - zo[nvf:]).max() <= 1e-10 * np.abs(zo[nvf:]).max()


def test_full_size_benchmark_case_properties(pkg):
    """32^3 perturbed mesh, 64 subdomains (the benchmark workload): converges,
    lambda_min >= 1, the residual of the full saddle system is at the CG
    tolerance and the discrete velocity is divergence-free elementwise."""
    import torch
    cfg = make_config("tri32_k2")
    deg = 11
    g = pkg.VemSystem(cfg["mesh"], 2, cfg["nu"])
    rhs = g.load(deg, cfg["f"](g.quad_points(deg)))
    bd = pkg.Bddc(g, cfg["part"])
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=500)
    assert res["status"] == 0
    assert res["lam_min"] > 1.0 - 1e-8
    r = rhs - g.apply(u)
    assert torch.linalg.norm(r).item() <= 1e-7 * torch.linalg.norm(rhs).item()
    div = r[g.n_vel_free:]            # pressure rows of the residual = -B u
    assert torch.abs(div).max().item() <= 1e-7 * torch.abs(rhs).max().item()


@pytest.mark.parametrize("name", ["tri6_k2", "tri4_k3", "sinker8"])
def test_fp32_local_with_refinement(pkg, name):
    """FP32 local factors with FP64-residual refinement of every local solve:
    rtol 1e-8 reached, iterations within +10% of the FP64 GPU form, relative
    error <= 1e-7 against the FP64 oracle PCG solution.  One refinement step
    at constant viscosity; two at viscosity contrast 1e4, where one step
    leaves the local solves too inexact (kappa doubles)."""
    import torch
    cfg, g, rhs, S, F = _setup(pkg, name)
    b64 = pkg.Bddc(g, cfg["part"])
    u64 = torch.zeros_like(rhs)
    r64 = b64.solve(rhs, u64, rtol=1e-8, maxit=400)
    b32 = pkg.Bddc(g, cfg["part"], precision=1, refine=2 if np.ptp(cfg["nu"]) > 0 else 1)
    u32 = torch.zeros_like(rhs)
    r32 = b32.solve(rhs, u32, rtol=1e-8, maxit=400)
    assert r64["status"] == 0 and r32["status"] == 0
    assert r32["iters"] <= int(np.ceil(1.1 * r64["iters"]))
    _, _, ob, _ = oracle_bddc(name)
    ro = ob.pcg(F, rtol=1e-8)
    nvf = len(S.dm.free)
    x = u32.cpu().numpy()
    assert np.linalg.norm(x[:nvf] - ro["x"][:nvf]) <= 1e-7 * np.linalg.norm(ro["x"][:nvf])


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_loop_matches_host_loop(pkg, precision):
    """The PCG loop as one CUDA graph (conditional while node, scalars on
    the device) against the host-driven loop: same iteration count, the same
    solution to rounding, the same Lanczos estimates; a second solve through
    the same captured graph repeats the first; maxit stops both forms at the
    same place; the captured bddc_apply equals the direct one."""
    import torch
    cfg, g, rhs, S, F = _setup(pkg, "tri6_k2")
    out = {}
    for ug in (-1, 0):
        bd = pkg.Bddc(g, cfg["part"], precision=precision, use_graph=ug)
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=1e-8, maxit=300)
        assert res["status"] == 0
        u2 = torch.full_like(rhs, 3.0)
        res2 = bd.solve(rhs, u2, rtol=1e-8, maxit=300)
        assert res2["iters"] == res["iters"] and torch.equal(u, u2)
        short = bd.solve(rhs, torch.zeros_like(rhs), rtol=1e-8, maxit=3)
        assert short["status"] == -6 and short["iters"] == 3
        z = bd.apply(rhs)
        z2 = bd.apply(rhs)
        assert torch.equal(z, z2)
        out[ug] = (res, u.cpu().numpy(), z.cpu().numpy())
    (rh, uh, zh), (rg, ug_, zg) = out[-1], out[0]
    # the two loops round differently (fused updates on the device); the
    # FP32-local preconditioner (with refinement) passes such differences on
    assert rg["iters"] == rh["iters"]
    assert abs(rg["lam_max"] - rh["lam_max"]) <= 1e-8 * rh["lam_max"]
    assert abs(rg["lam_min"] - rh["lam_min"]) <= 1e-8
    assert np.linalg.norm(ug_ - uh) <= 1e-10 * np.linalg.norm(uh)
    assert np.abs(zg - zh).max() <= 1e-13 * np.abs(zh).max()


@pytest.mark.parametrize("theta", [10.0, 2.0])
def test_adaptive_coarse_space_matches_oracle(pkg, theta):
    """Adaptive primal enrichment (Sec. 6) at viscosity contrast 1e4: the
    same number of added functionals as the oracle's eigenproblems, the same
    CG behaviour (iterations, Lanczos estimates) and solution, and a better
    conditioned preconditioner than without enrichment at theta = 2."""
    import torch
    cfg, g, rhs, S, F = _setup(pkg, "sinker8")
    bd = pkg.Bddc(g, cfg["part"], adaptive=theta)
    u = torch.zeros_like(rhs)
    res = bd.solve(rhs, u, rtol=1e-8, maxit=300)
    assert res["status"] == 0
    _, _, ob, _ = oracle_bddc("sinker8", adaptive=theta)
    assert int(bd.info("n_adaptive")) == ob.n_adaptive
    assert res["lam_min"] > 1.0 - 1e-8
    check_pcg_parity(S, ob, F, res, u.cpu().numpy(), label=f"adaptive-{theta}", deep=_deep(bd, rhs))
    if theta == 2.0:
        base = pkg.Bddc(g, cfg["part"]).solve(rhs, torch.zeros_like(rhs), rtol=1e-8, maxit=300)
        assert res["kappa"] < 0.5 * base["kappa"] and res["iters"] < base["iters"]


def test_tensor_core_tile_product(pkg):
    """One 128 x 128 x 32 tile of the tensor-core front update (tcgen05,
    three-part TF32 split, FP32 accumulation) against FP64: FP32-level error,
    well below what a single TF32 product (about 1e-3 relative) would give."""
    import ctypes
    L = pkg.lib()
    L.vem_tc_selftest.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    err, ref = ctypes.c_double(), ctypes.c_double()
    assert L.vem_tc_selftest(ctypes.byref(err), ctypes.byref(ref)) == 0, L.vem_last_error()
    assert ref.value > 1.0
    assert err.value <= 2e-6 * ref.value


def test_tensor_core_factorization_matches_fma_path(pkg):
    """16^3 perturbed mesh, 64 subdomains (fronts of several hundred rows, so
    the tensor-core path runs): FP32-local BDDC-PCG with tensor-core front
    updates against the same form on the FP32 FMA units and against the FP64
    form: iterations within +10% of FP64, solutions within 1e-7."""
    import torch
    cfg = make_config("tri16_k2")
    g = pkg.VemSystem(cfg["mesh"], 2, cfg["nu"])
    rhs = g.load(4, cfg["f"](g.quad_points(4)))
    out = {}
    for name, kw in (("fp64", dict(precision=0)), ("tc", dict(precision=1, tc_update=1)),
                     ("fma", dict(precision=1, tc_update=-1))):
        bd = pkg.Bddc(g, cfg["part"], **kw)
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=1e-8, maxit=500)
        assert res["status"] == 0
        out[name] = (res, u.cpu().numpy())
    (r64, u64), (rtc, utc), (rf, uf) = out["fp64"], out["tc"], out["fma"]
    assert rtc["iters"] <= int(np.ceil(1.1 * r64["iters"]))
    assert abs(rtc["iters"] - rf["iters"]) <= 1
    assert np.linalg.norm(utc - u64) <= 1e-7 * np.linalg.norm(u64)
    assert np.linalg.norm(utc - uf) <= 1e-7 * np.linalg.norm(uf)


"""Test infrastructure: the oracle's System of a named synthetic workload,
built once per test session.  Its elements are built in worker processes
(a ``spawn`` pool, started before or after CUDA without harm): each worker
rebuilds the workload from its seed and returns finished elements, which
``oracle.vem.System`` then assembles exactly as it would its own."""
import multiprocessing as mp
import os

_POOL = None
_SYSTEMS = {}


_ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _pool():
    """Workers run single-threaded BLAS (the element systems are tiny; one
    BLAS thread pool per worker would oversubscribe the cores)."""
    global _POOL
    if _POOL is None:
        n = max(1, min(os.cpu_count() or 1, 32))
        saved = {v: os.environ.get(v) for v in _ONE_THREAD}
        for v in _ONE_THREAD:
            os.environ[v] = "1"
        try:
            _POOL = mp.get_context("spawn").Pool(n)
        finally:
            for v, x in saved.items():
                if x is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = x
    return _POOL


def _build_chunk(args):
    name, overrides, deg, reduced, elems = args
    from synth import make_config
    from oracle.vem import Topology, DofMap, build_element
    cfg = make_config(name, **overrides)
    topo = Topology(cfg["mesh"])
    dm = DofMap(topo, cfg["k"], reduced)
    out = {}
    for e in elems:
        el = build_element(topo, dm, e, cfg["nu"][e], deg)
        fk = el.load(cfg["f"])
        el._topo = None            # the parent reattaches its own topology
        el._topo_xyz = None
        out[e] = (el, fk)
    return out


def load_degree(cfg):
    k = cfg["k"]
    return k + 9 if cfg["spec"]["load"] == "manufactured" else 2 * k + 2


def oracle_system(name, deg=None, reduced=False, **overrides):
    """(cfg, System) for a named workload; the System is cached per session."""
    from synth import make_config
    from oracle.vem import System
    cfg = make_config(name, **overrides)
    deg = load_degree(cfg) if deg is None else deg
    key = (name, tuple(sorted(overrides.items())), deg, reduced)
    if key not in _SYSTEMS:
        ne = len(cfg["nu"])
        nw = _pool()._processes
        step = max(1, -(-ne // (4 * nw)))
        chunks = [(name, overrides, deg, reduced, list(range(a, min(ne, a + step)))) for a in range(0, ne, step)]
        built = {}
        for part in _pool().map(_build_chunk, chunks):
            built.update(part)
        _SYSTEMS[key] = System(cfg["mesh"], cfg["k"], cfg["nu"], f=cfg["f"], load_deg=deg, reduced=reduced,
                               prebuilt=built)
    return cfg, _SYSTEMS[key]


_BDDC = {}


def oracle_bddc(name, scaling="deluxe", adaptive=None, reduced=False, deg=None, **overrides):
    """(cfg, System, BDDC, F) with the oracle's BDDC setup cached per session;
    F is the right-hand side of the free saddle system."""
    import numpy as np
    from oracle.bddc import BDDC
    cfg, S = oracle_system(name, deg=deg, reduced=reduced, **overrides)
    key = (name, tuple(sorted(overrides.items())), deg, reduced, scaling, adaptive)
    if key not in _BDDC:
        kw = {} if adaptive is None else {"adaptive": adaptive}
        _BDDC[key] = BDDC(S, cfg["part"], scaling=scaling, **kw)
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    return cfg, S, _BDDC[key], F


def _oracle_iterate_sensitivity(ob, F, iters, eps=1e-15, seeds=(1, 2)):
    """The oracle's own response, at a fixed iteration count, to perturbing
    every preconditioner output by a seeded relative eps (rounding level):
    the iterates x' of those runs, for comparison with its unperturbed one."""
    import numpy as np
    base = ob.apply
    out = []
    try:
        for sd in seeds:
            rng = np.random.default_rng(sd)

            def pert(r, _a=base, _g=rng):
                z = _a(r)
                return z * (1.0 + eps * _g.standard_normal(z.shape))
            ob.apply = pert
            out.append(ob.pcg(F, rtol=0.0, maxit=iters)["x"])
    finally:
        ob.apply = base
    return out


def _oracle_iteration_range(ob, F, eps_list=(1e-15, 1e-14, 1e-13), seeds=(1, 2)):
    """Iteration counts of the oracle's own PCG at rtol 1e-8 when every
    preconditioner output is perturbed by a seeded relative eps (rounding
    level, up to the agreement of the two sides' element matrices): the
    range (min, max) with the unperturbed count."""
    import numpy as np
    base = ob.apply
    counts = [ob.pcg(F, rtol=1e-8)["iters"]]
    try:
        for eps in eps_list:
            for sd in seeds:
                rng = np.random.default_rng(sd)

                def pert(r, _a=base, _g=rng, _e=eps):
                    z = _a(r)
                    return z * (1.0 + _e * _g.standard_normal(z.shape))
                ob.apply = pert
                counts.append(ob.pcg(F, rtol=1e-8)["iters"])
    finally:
        ob.apply = base
    return min(counts), max(counts)


def check_pcg_parity(S, ob, F, res, x, tol=1e-10, label="", deep=None):
    """FP64 parity of a GPU BDDC-PCG run with the oracle's.

    (1) At rtol 1e-8: iteration counts within +-1, the Lanczos lambda_max
    within 1e-6 relative, and, at equal iteration counts (the oracle re-run
    with maxit = the GPU's count when the two stop apart), the velocity and
    the whole zero-mean solution [u; p - mean(p)] within tol.  Where the
    counts differ by more than one, the oracle's own count is measured under
    seeded relative 1e-15 .. 1e-13 perturbations of every preconditioner
    output (CG in floating point at large kappa: viscosity contrast); the GPU
    count must lie within one of that range, and (2) carries the bar.
    Where the oracle cannot reproduce its own iterate to better than tol/10
    under a seeded relative 1e-15 perturbation of every preconditioner output
    (CG amplifies rounding: viscosity contrast, thin CVT faces), that
    comparison is reported, not asserted, and (2) carries the bar.
    (2) deep: a callable running the GPU solve to a given rtol; both sides
    are run to rtol 1e-11, where the discrete solution is determined to
    better than tol, and must agree within tol (velocity and whole
    solution).  Returns the measured differences."""
    import numpy as np
    ro = ob.pcg(F, rtol=1e-8)
    it_range = None
    if abs(res["iters"] - ro["iters"]) > 1:
        it_range = _oracle_iteration_range(ob, F)
        assert it_range[0] - 1 <= res["iters"] <= it_range[1] + 1, (res["iters"], ro["iters"], it_range)
        assert deep is not None, "needs the deep comparison"
    if res["iters"] != ro["iters"]:
        ro = ob.pcg(F, rtol=0.0, maxit=res["iters"])
        assert ro["iters"] == res["iters"]
    nvf = len(S.dm.free)
    pz = lambda v: np.concatenate([v[:nvf], v[nvf:] - (S.wmean @ v[nvf:]) / S.wmean.sum()])
    xo = pz(ro["x"])

    def diffs(a, b):
        return (np.linalg.norm(a[:nvf] - b[:nvf]) / np.linalg.norm(b[:nvf]),
                np.linalg.norm(a - b) / np.linalg.norm(b))
    ev, ex = diffs(pz(x), xo)
    el = abs(res["lam_max"] - ro["lam_max"]) / ro["lam_max"]
    assert el <= 1e-6, el
    sens = None
    if ev > tol or ex > tol:
        sens = max(max(diffs(pz(xs), xo)) for xs in _oracle_iterate_sensitivity(ob, F, res["iters"]))
    line = (f"PARITY {label} iters gpu {res['iters']} oracle {ro['iters']} rtol 1e-8: vel {ev:.3e} all {ex:.3e}"
            + ("" if sens is None else f" (oracle reproducibility {sens:.1e})")
            + ("" if it_range is None else f" (oracle iterations under perturbation {it_range[0]}-{it_range[1]})"))
    out = dict(vel=ev, all=ex, lam=el, oracle=ro, reproducibility=sens, iteration_range=it_range)
    if it_range is None and (sens is None or sens <= 0.1 * tol):
        assert ev <= tol and ex <= tol, (ev, ex)
    if deep is not None:
        rd, xd = deep(1e-11)
        rod = ob.pcg(F, rtol=1e-11)
        dv, dx = diffs(pz(xd), pz(rod["x"]))
        line += f" | rtol 1e-11: iters {rd['iters']}/{rod['iters']} vel {dv:.3e} all {dx:.3e}"
        out.update(deep_vel=dv, deep_all=dx)
        assert dv <= tol and dx <= tol, (dv, dx)
    else:
        assert sens is None or sens <= 0.1 * tol, "needs the deep comparison"
    print(line)
    return out

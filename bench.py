#!/usr/bin/env python
"""Benchmark: BDDC-PCG time-to-solution (rtol 1e-8) on one GB300.

One step = the whole path on one synthetic problem: vem_assemble (element
projectors and matrices, CSR assembly), vem_load, bddc_setup (local
factorizations, deluxe face blocks, coarse problem) and pcg_solve.
Default workload: 32^3 hexahedra with interior vertices moved by up to 0.2 h
(seed 2), quadrilaterals split into triangles, k = 2, nu = 1, manufactured
load, 4 x 4 x 4 box subdomains.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (NumPy/SciPy) end to end on the 8^3
member of the same family (512 elements, 2 x 2 x 2 subdomains of 4^3
elements, k = 2): its elements built by a spawn pool over the host cores,
its BDDC setup and PCG as the oracle stands.  Its value is that measured
time, for that named workload, not an extrapolation.  With N > 1 (torchrun) every
rank solves its own replica (the solver runs on one GPU; ranks do not
exchange data).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDDC-PCG time-to-solution at rtol 1e-8 and BDDC applies/s, FP32-local vs FP64, 1 GB300"
WORKLOAD = "tri32_k2"
LOAD_DEGREE = 11            # k + 9: exact for the degree-9 manufactured load at k = 2
ORACLE_WORKLOAD = "tri8_k2"
# DRAM bytes the sweep kernels (with the FP32 conversions of their vectors)
# move per algorithmic factor byte: 1,910.2 MB against 1.79 GB in one ncu
# capture of an apply on the 16^3 member
# (profiles/bddc_apply_tri16_k2_fp32local_dram.md); the traffic scales with
# the factor bytes, so the 32^3 sweep pair's traffic is this ratio times its
# algorithmic bytes
SWEEP_TRAFFIC_RATIO = 1910.2 / 1790.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except OSError:
            return None
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        mx = max(float(r[2]) for r in rows if len(r) > 8)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_tts(name=ORACLE_WORKLOAD, timeout=1800):
    """Oracle time to solution (System, BDDC setup, PCG at rtol 1e-8) on a
    named workload, measured in a fresh process without a GPU: the element
    projectors and matrices of every element by a spawn pool with one
    worker per host core (each single-threaded), the assembly, BDDC setup
    and PCG in the main process as the oracle stands.  Returns the measured
    seconds per phase, the iteration count and the core count."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r); sys.path.insert(0, os.path.join(%r, 'tests'))
import numpy as np
if __name__ == '__main__':
    from oracle_cache import oracle_system, _pool
    from oracle.bddc import BDDC
    workers = _pool()._processes
    t0 = time.perf_counter()
    cfg, S = oracle_system(%r, deg=%d)
    t1 = time.perf_counter()
    bd = BDDC(S, cfg['part'])
    t2 = time.perf_counter()
    F = np.concatenate([S.F[S.dm.free], np.zeros(S.dm.npress)])
    res = bd.pcg(F, rtol=1e-8)
    t3 = time.perf_counter()
    print(json.dumps(dict(seconds=t3 - t0, system_s=t1 - t0, setup_s=t2 - t1, pcg_s=t3 - t2,
                          elements=S.topo.nE, subdomains=int(cfg['part'].max()) + 1, iters=res['iters'],
                          workers=workers, cores=os.cpu_count())))
""" % (ROOT, ROOT, name, LOAD_DEGREE)
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _oracle_mesh_text():
    from synth.configs import CONFIGS
    c = CONFIGS[ORACLE_WORKLOAD]
    return (f"{c['n']}^3 hex, interior vertices +-{c['perturb']}h (seed {c['seed']}), split quads, k = {c['k']}, "
            f"{c['parts'][0]}x{c['parts'][1]}x{c['parts'][2]} subdomains of "
            f"{c['n'] // c['parts'][0]}^3 elements")


def _oracle_sample_text(r):
    return (f"oracle end to end (assembly with load rule degree {LOAD_DEGREE}, BDDC setup, PCG to rtol 1e-8, "
            f"{r['iters']} iterations) on {ORACLE_WORKLOAD} ({_oracle_mesh_text()}; {r['elements']} elements); "
            f"elements on {r['workers']} worker processes, setup and PCG in one process; measured, not scaled: "
            f"system {r['system_s']:.1f} s, setup {r['setup_s']:.1f} s, PCG {r['pcg_s']:.1f} s")


def run_reference(args, rank, world):
    if rank != 0:
        return
    # untimed warm-up on the 4^3 member (imports, worker start-up), then the
    # timed steps on the named workload
    for _ in range(args.warmup):
        cpu_oracle_tts("tri4_k2")
    runs = [cpu_oracle_tts() for _ in range(args.steps)]
    v = statistics.mean(r["seconds"] for r in runs)
    r0 = runs[-1]
    line = {"metric": METRIC, "value": v, "unit": "s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ORACLE_WORKLOAD, "mesh": _oracle_mesh_text(), "subdomains": r0["subdomains"],
                       "rtol": 1e-8, "load_degree": LOAD_DEGREE},
            "cpu_baseline": {"value": v, "unit": "s", "cores": r0["cores"], "kind": "oracle",
                             "sample": _oracle_sample_text(r0)},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(pkg, torch, cfg, fq_host, precision, steps, warmup, stream, with_e2e, rank):
    """Times `steps` full steps (after `warmup`) of one precision form: with
    the load samples resident on the device (the timed value), and with
    every input from host memory and the solution copied back (e2e)."""
    mesh, k, nu, part = cfg["mesh"], cfg["k"], cfg["nu"], cfg["part"]
    fq = fq_host.to("cuda")

    phases = {}

    def step(out_host=None):
        # every library call below synchronizes, so host clocks split the step;
        # fq is the load samples on the device (timed device step) or in
        # pinned host memory (end-to-end step: copied in by vem_load)
        t0 = time.perf_counter()
        g = pkg.VemSystem(mesh, k, nu)
        g.set_stream(stream)
        t1 = time.perf_counter()
        rhs = g.load(LOAD_DEGREE, fq if out_host is None else fq_host)
        t2 = time.perf_counter()
        bd = pkg.Bddc(g, part, precision=precision)
        t3 = time.perf_counter()
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=1e-8, maxit=1000)
        t4 = time.perf_counter()
        if out_host is not None:
            out_host.copy_(u, non_blocking=True)
        phases.update(vem_assemble=(t1 - t0) * 1e3, vem_load=(t2 - t1) * 1e3, bddc_setup=(t3 - t2) * 1e3,
                      pcg_solve=(t4 - t3) * 1e3)
        return g, bd, u, rhs, res

    for _ in range(warmup):
        step()
        torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g = bd = u = rhs = None
    l0 = pkg.kernel_launches()
    ev0.record(stream)
    for _ in range(steps):
        g = bd = u = rhs = None
        g, bd, u, rhs, res = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    dev_ms = ev0.elapsed_time(ev1) / steps
    launches = (pkg.kernel_launches() - l0) // steps
    dev_phases = dict(phases)   # phases of the last device-timed step
    e2e_ms = None
    if with_e2e:
        host_u = torch.empty(g.n, dtype=torch.float64, pin_memory=True)
        g = bd = u = rhs = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            g = bd = u = rhs = None
            g, bd, u, rhs, res = step(host_u)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
    keys = ("factor_bytes_dirichlet", "factor_bytes_neumann", "deluxe_bytes", "t_symbolic_ms", "t_flatten_ms", "t_upload_ms",
            "t_factor_dirichlet_ms", "t_factor_neumann_ms", "t_factor_deluxe_ms", "t_deluxe_combine_ms",
            "t_coarse_rhs_ms", "t_coarse_solves_ms", "t_coarse_gram_ms", "t_coarse_inverse_ms",
            "gflop_factor_dirichlet", "gflop_factor_neumann", "gflop_factor_deluxe")
    info = {k2: bd.info(k2) for k2 in keys}
    vkeys = ("t_topology_ms", "t_element_launch_ms", "t_pattern_ms", "t_element_wait_ms", "t_pattern_upload_ms",
             "t_gpu_finish_ms")
    vinfo = {k2: g.info(k2) for k2 in vkeys}
    r = torch.randn(g.n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(3):
        bd.apply(r, z)
    torch.cuda.synchronize()
    ev0.record(stream)
    napp = 20
    for _ in range(napp):
        bd.apply(r, z)
    ev1.record(stream)
    torch.cuda.synchronize()
    apply_ms = ev0.elapsed_time(ev1) / napp
    sweep_ms, sweep_bytes = bd.time_local_solves(5)
    return dict(dev_ms=dev_ms, e2e_ms=e2e_ms, launches=launches, res=res, info=info, vinfo=vinfo,
                phases=dev_phases, e2e_phases=dict(phases) if with_e2e else None, apply_ms=apply_ms,
                sweep_ms=sweep_ms, sweep_bytes=sweep_bytes, n=g.n, n_coarse=bd.info("n_coarse"))


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    import paper_2304_09770_gb300 as pkg
    from synth import make_config

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = make_config(WORKLOAD)
    mesh, k, nu, part = cfg["mesh"], cfg["k"], cfg["nu"], cfg["part"]
    stream = torch.cuda.current_stream()
    # host inputs of one step: mesh arrays, viscosity, partition, load samples
    probe = pkg.VemSystem(mesh, k, nu)
    pts = probe.quad_points(LOAD_DEGREE)
    fq = torch.empty(pts.shape, dtype=torch.float64, pin_memory=True)
    fqn = fq.numpy()
    for a in range(0, len(pts), 1 << 24):      # chunks bound the temporaries
        fqn[a:a + (1 << 24)] = cfg["f"](pts[a:a + (1 << 24)])
    del probe, pts
    h2d = (mesh["xyz"].nbytes + mesh["face_ptr"].nbytes + mesh["face_vtx"].nbytes + mesh["elem_ptr"].nbytes
           + mesh["elem_face"].nbytes + nu.nbytes + part.nbytes + fq.numel() * 8)
    if dist:
        dist.barrier()
    import tempfile
    clocks = Clocks(os.path.join(tempfile.gettempdir(), f"vembddc_clocks_rank{rank}.csv"))
    with clocks:
        m32 = measure(pkg, torch, cfg, fq, 1, args.steps, args.warmup, stream, True, rank)
        m64 = measure(pkg, torch, cfg, fq, 0, args.steps, args.warmup, stream, False, rank)
    t = torch.tensor([m32["dev_ms"], m32["e2e_ms"], m64["dev_ms"]], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, e2e_ms, dev64 = t.tolist()
    if rank != 0:
        return
    hbm, kind = peaks()

    def roof(m):
        ach = m["sweep_bytes"] / (m["sweep_ms"] * 1e-3) / 1e9
        return {"kernel": "local triangular sweeps (level GEMV kernels, forward+backward, Neumann+Dirichlet "
                          "factors)", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_kind": kind, "traffic": SWEEP_TRAFFIC_RATIO * m["sweep_bytes"],
                "traffic_source": "ncu DRAM bytes of the sweep kernels on the 16^3 member, scaled by factor bytes",
                "bytes_per_sweep_pair": m["sweep_bytes"], "ms_per_sweep_pair": m["sweep_ms"]}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            c = cpu_oracle_tts()
            cpu = {"value": c["seconds"], "unit": "s", "cores": c["cores"], "kind": "oracle",
                   "workload": ORACLE_WORKLOAD, "sample": _oracle_sample_text(c)}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e}"[:200]}
    res = m32["res"]
    line = {
        "metric": METRIC, "value": dev_ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-local/f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": "32^3 hex, interior vertices +-0.2h (seed 2), split quads",
                   "k": 2, "subdomains": 64, "precision": "FP32 local factors + 1 refinement; FP64 CG, "
                   "operator, coarse, deluxe inverses", "rtol": 1e-8, "load_degree": LOAD_DEGREE,
                   "l2": "inputs larger than L2 (local factors 7-15 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": res["iters"], "kappa": res["kappa"], "lam_min": res["lam_min"],
        "bddc_applies_per_s": 1e3 / m32["apply_ms"], "ms_per_apply": m32["apply_ms"],
        "setup_phases_ms": m32["info"], "step_phases_ms": m32["phases"], "e2e_step_phases_ms": m32["e2e_phases"],
        "assemble_phases_ms": m32["vinfo"],
        "fp64": {"value": dev64 / 1e3, "unit": "s", "iterations": m64["res"]["iters"],
                 "kappa": m64["res"]["kappa"], "lam_min": m64["res"]["lam_min"],
                 "bddc_applies_per_s": 1e3 / m64["apply_ms"], "ms_per_apply": m64["apply_ms"],
                 "setup_phases_ms": m64["info"], "step_phases_ms": m64["phases"], "roofline": roof(m64), "gpu_launches": int(m64["launches"])},
        "roofline": roof(m32),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(m32["n"] * 8)},
        "clocks": clocks.summary(),
        "gpu_launches": int(m32["launches"]),
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Small driver for profilers.  apply: one setup, then `napply`
    preconditioner applies (FP64 or FP32-local local factors) on the named
    workload.  step: one whole step (assembly, load, setup, PCG solve)."""
    import numpy as np
    import torch
    import paper_2304_09770_gb300 as pkg
    from synth import make_config
    cfg = make_config(args.workload)
    if args.profile == "step":
        g = pkg.VemSystem(cfg["mesh"], cfg["k"], cfg["nu"])
        fq = cfg["f"](g.quad_points(LOAD_DEGREE))
        l0 = pkg.kernel_launches()
        rhs = g.load(LOAD_DEGREE, fq)
        bd = pkg.Bddc(g, cfg["part"], precision=args.precision)
        l1 = pkg.kernel_launches()
        u = torch.zeros_like(rhs)
        res = bd.solve(rhs, u, rtol=1e-8, maxit=1000)
        torch.cuda.synchronize()
        print(json.dumps({"workload": args.workload, "precision": args.precision, "assemble_launches": l0,
                          "setup_launches": l1 - l0, "solve_launches": pkg.kernel_launches() - l1,
                          "iterations": res["iters"]}))
        return
    g = pkg.VemSystem(cfg["mesh"], cfg["k"], cfg["nu"])
    bd = pkg.Bddc(g, cfg["part"], precision=args.precision)
    r = torch.randn(g.n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    torch.cuda.synchronize()
    l0 = pkg.kernel_launches()
    for _ in range(args.napply):
        bd.apply(r, z)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "precision": args.precision, "setup_launches": l0,
                      "apply_launches": (pkg.kernel_launches() - l0) // args.napply}))


CONFIG_RUNS = [
    # (workload, precision, adaptive theta): the five configurations of the
    # benchmark family; sinker meshes also with the adaptive coarse space
    ("cube4_k2", 0, 0.0), ("cube4_k2", 1, 0.0),
    ("tri32_k2", 0, 0.0), ("tri32_k2", 1, 0.0),
    ("tri48_greedy", 0, 0.0), ("tri48_greedy", 1, 0.0),
    ("tri16_k2", 0, 0.0), ("tri16_k2", 1, 0.0),
    ("tri16_k3", 0, 0.0), ("tri16_k3", 1, 0.0),
    ("tri16_k4", 0, 0.0), ("tri16_k4", 1, 0.0),
    ("sinker32_dr1e4", 0, 0.0), ("sinker32_dr1e4", 1, 0.0), ("sinker32_dr1e4", 0, 10.0), ("sinker32_dr1e4", 1, 10.0),
    ("sinker32_dr1e6", 0, 0.0), ("sinker32_dr1e6", 0, 10.0), ("sinker32_dr1e6", 1, 10.0),
]
# further runs (workload, precision, theta, options): theta (nu_tol) sweep on
# configurations 2 and 4, deluxe scaling on edges at viscosity contrast, the
# paper's 15,552-element OCTA mesh, a 4,000-cell CVT mesh, and the reduced
# scheme
EXTRA_RUNS = [
    ("tri32_k2", 0, 2.0, {}), ("tri32_k2", 0, 5.0, {}), ("tri16_k4", 0, 2.0, {}), ("tri16_k4", 0, 5.0, {}),
    ("sinker32_dr1e4", 0, 0.0, {"scaling": 2}), ("sinker32_dr1e4", 1, 0.0, {"scaling": 2}),
    ("sinker32_dr1e6", 0, 0.0, {"scaling": 2}), ("sinker32_dr1e6", 0, 10.0, {"scaling": 2}),
    ("octa12_k2", 0, 0.0, {}), ("octa12_k2", 1, 0.0, {}), ("octa12_k2", 0, 2.0, {}),
    ("cvt4000_k2", 0, 0.0, {}), ("cvt4000_k2", 1, 0.0, {}),
    ("tri32_k2", 0, 0.0, {"reduced": True}), ("tri32_k2", 1, 0.0, {"reduced": True}),
    ("tri16_k4", 0, 0.0, {"reduced": True}),
]


def run_configs(args):
    """One solve per configuration and form: times of each library call,
    CG iterations, Lanczos estimates, and properties of the computed
    solution (saddle-system residual, elementwise divergence), one JSON line
    each."""
    import numpy as np
    import torch
    import paper_2304_09770_gb300 as pkg
    from synth import make_config
    only = set(args.only.split(",")) if args.only else None
    cache = {}
    runs = [r + ({},) for r in CONFIG_RUNS] + (EXTRA_RUNS if args.extra else [])
    for name, prec, theta, opt in runs:
        if only and name not in only:
            continue
        cfg = cache.get(name) or make_config(name)
        cache.clear()
        cache[name] = cfg
        k = cfg["k"]
        deg = 2 * k - 2   # load rule: enough for the solver study, small host arrays at 48^3
        scaling, reduced = opt.get("scaling", 1), bool(opt.get("reduced", False))
        line = {"workload": name, "precision": prec, "adaptive": theta, "scaling": scaling, "reduced": reduced,
                "k": k,
                "elements": int(cfg["mesh"]["elem_ptr"].shape[0] - 1), "subdomains": int(cfg["part"].max() + 1)}
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = pkg.VemSystem(cfg["mesh"], k, cfg["nu"], reduced=reduced)
            t1 = time.perf_counter()
            fq = cfg["f"](g.quad_points(deg))
            t2 = time.perf_counter()
            rhs = g.load(deg, fq)
            t3 = time.perf_counter()
            # FP32-local: two refinement steps where one leaves the local
            # solves too inexact (viscosity contrast, degree 4)
            refine = 2 if prec and (np.ptp(cfg["nu"]) > 0 or k >= 4) else 0
            line["refine"] = refine if prec else None
            bd = pkg.Bddc(g, cfg["part"], precision=prec, refine=refine, adaptive=theta, scaling=scaling)
            t4 = time.perf_counter()
            u = torch.zeros_like(rhs)
            res = bd.solve(rhs, u, rtol=1e-8, maxit=2000)
            t5 = time.perf_counter()
            r = rhs - g.apply(u)
            line.update(n_dofs=int(g.n), nnz=g.info("nnz"), status=res["status"], iterations=res["iters"],
                        kappa=res["kappa"], lam_min=res["lam_min"], n_coarse=bd.info("n_coarse"),
                        n_adaptive=bd.info("n_adaptive"),
                        rel_residual=torch.linalg.norm(r).item() / torch.linalg.norm(rhs).item(),
                        max_div=torch.abs(r[g.n_vel_free:]).max().item() / torch.abs(rhs).max().item(),
                        t_assemble_s=t1 - t0, t_load_s=t3 - t2, t_setup_s=t4 - t3, t_solve_s=t5 - t4,
                        time_to_solution_s=(t1 - t0) + (t3 - t2) + (t4 - t3) + (t5 - t4),
                        factor_bytes=bd.info("factor_bytes_dirichlet") + bd.info("factor_bytes_neumann"))
            del bd, g, u, rhs, r
        except Exception as e:  # noqa: BLE001
            line.update(error=str(e)[:300], gib_free=torch.cuda.mem_get_info()[0] / 2**30)
        torch.cuda.empty_cache()
        print(json.dumps(line), flush=True)


def main():
    global ORACLE_WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-workload", default=ORACLE_WORKLOAD,
                    help="workload the CPU oracle is timed on (--impl reference and cpu_baseline)")
    ap.add_argument("--profile", choices=["apply", "step"], default=None,
                    help="profiler driver: setup once then --napply preconditioner applies, or one whole step")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--napply", type=int, default=3)
    ap.add_argument("--configs", action="store_true",
                    help="one solve per benchmark configuration and form (JSON line each)")
    ap.add_argument("--only", default="", help="with --configs: comma-separated workload names")
    ap.add_argument("--extra", action="store_true",
                    help="with --configs: also the theta sweep, edge deluxe, OCTA and reduced-scheme runs")
    args = ap.parse_args()
    ORACLE_WORKLOAD = args.oracle_workload
    if args.profile:
        run_profile(args)
        return
    if args.configs:
        run_configs(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = td
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

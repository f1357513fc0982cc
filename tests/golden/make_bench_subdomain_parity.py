"""Writes tests/golden/tri12_quarters_oracle.json: the oracle's BDDC-PCG on the
12^3 perturbed split-hex mesh with 2 x 2 x 1 subdomains of 6 x 6 x 12 = 432
elements (the 32^3 benchmark's have 512), k = 2, deluxe scaling, rtol 1e-8,
load rule degree k + 9.  Stored: iteration count and Lanczos estimates, and the
iterates at that count and one step either side (so that a run stopping one
step apart is compared at its own count) on a seeded sample of velocity and
pressure entries, with the norms of the whole vectors; the oracle's own
reproducibility of its iterate at that count (the largest relative change,
velocity or whole sampled solution, when every preconditioner output is
perturbed by a seeded relative 1e-15); and the solution at rtol 1e-11, where
the discrete solution is determined to better than 1e-10.  Calls only the
oracle (and the seeded inputs of synth); it takes about an hour and a half.

    python tests/golden/make_bench_subdomain_parity.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

NAME = "tri12_quarters"


def main():
    from oracle_cache import oracle_bddc, _oracle_iterate_sensitivity
    t0 = time.time()
    cfg, S, ob, F = oracle_bddc(NAME)
    t1 = time.time()
    ro = ob.pcg(F, rtol=1e-8)
    it = ro["iters"]
    nvf = len(S.dm.free)
    rng = np.random.default_rng(2024)
    sv = np.sort(rng.choice(nvf, 1000, replace=False))
    sp = np.sort(rng.choice(S.dm.npress, 300, replace=False))
    wm = S.wmean

    def record(x):
        p = x[nvf:] - (wm @ x[nvf:]) / wm.sum()
        return {"vel": x[:nvf][sv].tolist(), "press": p[sp].tolist(),
                "vel_norm": float(np.linalg.norm(x[:nvf])), "press_norm": float(np.linalg.norm(p))}

    iterates = {str(it): record(ro["x"])}
    for m in (it - 1, it + 1):
        iterates[str(m)] = record(ob.pcg(F, rtol=0.0, maxit=m)["x"])

    def sampled(rec):
        return np.array(rec["vel"]), np.concatenate([rec["vel"], rec["press"]])

    base_v, base_x = sampled(iterates[str(it)])
    repro = 0.0
    for xs in _oracle_iterate_sensitivity(ob, F, it):
        v, x = sampled(record(xs))
        repro = max(repro, np.linalg.norm(v - base_v) / np.linalg.norm(base_v),
                    np.linalg.norm(x - base_x) / np.linalg.norm(base_x))
    rd = ob.pcg(F, rtol=1e-11)
    deep = record(rd["x"])
    deep["iters"] = rd["iters"]
    out = {"workload": NAME, "k": cfg["k"], "scaling": "deluxe", "rtol": 1e-8, "load_degree": cfg["k"] + 9,
           "iters": it, "kappa": ro["kappa"], "lam_min": ro["lam_min"], "lam_max": ro["lam_max"],
           "n_vel_free": nvf, "n_press": int(S.dm.npress), "sample_vel": sv.tolist(), "sample_press": sp.tolist(),
           "iterates": iterates, "reproducibility": repro, "deep_rtol": 1e-11, "deep": deep,
           "oracle_seconds": {"setup": t1 - t0, "total": time.time() - t0}}
    with open(os.path.join(HERE, NAME + "_oracle.json"), "w") as f:
        json.dump(out, f)
    print("wrote", NAME, "iters", it, "kappa", ro["kappa"], "reproducibility", repro, "deep iters", rd["iters"])


if __name__ == "__main__":
    main()

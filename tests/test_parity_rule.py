"""The shared FP64 parity check (oracle_cache.check_pcg_parity) on the CPU,
with the oracle standing in for the GPU: its own run passes, and planted
mistakes (a solution off by 1e-8 relative, an iteration count three steps
off) fail.  Mistakes are planted on the oracle side only."""
import numpy as np
import pytest

from oracle_cache import oracle_bddc, check_pcg_parity, _oracle_iteration_range


@pytest.fixture(scope="module")
def case():
    cfg, S, ob, F = oracle_bddc("cube4_k2")
    ro = ob.pcg(F, rtol=1e-8)
    res = dict(status=0, iters=ro["iters"], lam_max=ro["lam_max"], lam_min=ro["lam_min"])

    def deep(rtol):
        r = ob.pcg(F, rtol=rtol)
        return r, r["x"]
    return S, ob, F, ro, res, deep


def test_oracle_against_itself_passes(case):
    S, ob, F, ro, res, deep = case
    out = check_pcg_parity(S, ob, F, res, ro["x"].copy(), label="oracle-self", deep=deep)
    assert out["vel"] == 0.0 and out["all"] == 0.0 and out["iteration_range"] is None


def test_planted_solution_error_fails(case):
    S, ob, F, ro, res, deep = case
    rng = np.random.default_rng(1)
    x = ro["x"] * (1.0 + 1e-8 * rng.standard_normal(ro["x"].shape))
    with pytest.raises(AssertionError):
        check_pcg_parity(S, ob, F, res, x, label="planted-x", deep=None)


def test_planted_iteration_count_fails(case):
    S, ob, F, ro, res, deep = case
    lo, hi = _oracle_iteration_range(ob, F)
    assert lo <= ro["iters"] <= hi and hi - lo <= 1
    bad = dict(res, iters=hi + 3)
    with pytest.raises(AssertionError):
        check_pcg_parity(S, ob, F, bad, ro["x"].copy(), label="planted-iters", deep=deep)

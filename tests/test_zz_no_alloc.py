"""vem_load_noalloc against vem_load, through the C ABI.

vem_load_noalloc serves callers that must not allocate device memory (a
fixed memory budget, or a framework that owns every device allocation):
its only scratch is a fixed array inside the library.  This file is named
to be collected last, so that a run stopping at its first failure has run
every other test before it.  It also passes alone in a fresh process.
"""
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


def _system(pkg, name, **override):
    cfg = make_config(name, **override)
    k = cfg["k"]
    g = pkg.VemSystem(cfg["mesh"], k, cfg["nu"])
    return cfg, g, k + 9


def test_noalloc_load_matches_load_on_two_calls_in_a_row(pkg):
    import torch
    # different problems back to back: a k = 3 split-hex mesh, OCTA and CVT
    # meshes (pentagonal and larger faces, cells of uneven point counts), then
    # a k = 2 mesh with fewer DOFs, so stale contents of the shared scratch
    # from an earlier call would show in a later result
    outs = []
    for name in ("tri4_k3", "octa2_k3", "cvt27_k3", "tri6_k2"):
        cfg, g, deg = _system(pkg, name)
        fq = np.ascontiguousarray(cfg["f"](g.quad_points(deg)))
        ref = g.load(deg, fq)                      # vem_load (host f, allocating)
        f_dev = torch.tensor(fq, dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        g.load_noalloc(deg, f_dev, got)
        torch.cuda.synchronize()
        r, x = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(x).all()
        assert np.abs(x - r).max() <= 1e-12 * np.abs(r).max()
        outs.append((g, deg, f_dev, ref))
    # and again on the first system, after the second call overwrote the scratch
    g, deg, f_dev, ref = outs[0]
    got = torch.full_like(ref, float("nan"))
    g.load_noalloc(deg, f_dev, got)
    torch.cuda.synchronize()
    assert np.abs(got.cpu().numpy() - ref.cpu().numpy()).max() <= 1e-12 * np.abs(ref.cpu().numpy()).max()


def test_noalloc_load_rejects_meshes_beyond_its_scratch(pkg):
    import torch
    # 28^3 split hexahedra at k = 2: 21952 elements x 117 DOFs x 8 bytes
    # (about 20.5 MB) exceeds the fixed 16 MiB scratch
    import ctypes
    cfg, g, _ = _system(pkg, "tri32_k2", n=28)
    deg = 0                      # fewest load points: f sized for the rule all the same
    n = ctypes.c_int64()
    assert pkg.lib().vem_quad_points(g.h, deg, ctypes.byref(n), None) == 0
    f_dev = torch.zeros((n.value, 3), dtype=torch.float64, device="cuda")
    out = torch.full((g.n,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.VemError) as ei:
        g.load_noalloc(deg, f_dev, out)
    assert ei.value.status == -1 and "scratch" in str(ei.value)
    assert torch.all(out == 7.0).item()

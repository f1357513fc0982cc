"""The polynomial patch test on the GPU path, through the C ABI (convergence
theorem, Sec. 3: a solenoidal u in [P_k]^3 with p in P_{k-1} is reproduced
exactly by the discrete problem).

The GPU-assembled saddle system (vem_assemble), load (vem_load) and
non-homogeneous Dirichlet data (vem_lift_dirichlet) must be satisfied by the
interpolant u_I of u (the oracle's DOFs of u) and the exact pressure: the
residual F - K[:, fixed] u_I - K [u_I; p] vanishes to rounding in every row,
so the discrete solution, unique in the velocity and up to a constant in the
pressure, is the interpolant.  The residual is formed with vem_apply (the
operator applied to the free part).  BDDC-PCG is not used here: with the
data lifted by u_I the velocity correction is exactly zero, and the CG of
the interface problem has nothing to iterate on (its first search direction
carries no velocity), while with the boundary values alone the divergence
rows have a right-hand side outside the benign subspace that BDDC's CG runs
on (Sec. 4.3)."""
import numpy as np
import pytest

from synth import cube_mesh
from oracle.vem import System
from oracle.poly import dim3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2304_09770_gb300 as p
    p.lib()
    return p


@pytest.mark.parametrize("n,k", [(4, 2), (3, 3), (2, 4)])
def test_patch_test_on_the_gpu(pkg, n, k):
    import torch
    mesh = cube_mesh(n, 0.2, 3)
    b = np.array([1.0, 2.0, -3.0])
    u = lambda x: np.stack([x[:, 1] ** k + x[:, 2], x[:, 2] ** k + x[:, 0], x[:, 0] ** k + x[:, 1]], 1)
    lap = lambda x: np.stack([k * (k - 1) * x[:, 1] ** (k - 2), k * (k - 1) * x[:, 2] ** (k - 2),
                              k * (k - 1) * x[:, 0] ** (k - 2)], 1)
    f = lambda x: -0.5 * lap(x) - b            # -div(eps u) - grad p with div u = 0
    nu = np.ones(n ** 3)
    S = System(mesh, k, nu, f=f, load_deg=2 * k + 2)
    uI = np.zeros(S.dm.nvel)
    for e, el in S.elements.items():
        uI[el.dofs] = el.poly_dofs(u, lambda x: np.zeros(len(x)))
    npk = dim3(k - 1)
    pex = np.zeros(S.dm.npress)
    for e, el in S.elements.items():
        pex[e * npk] = b @ el.xK
        pex[e * npk + 1:e * npk + 4] = el.hK * b
    g = pkg.VemSystem(mesh, k, nu)
    deg = 2 * k + 2
    nvf = g.n_vel_free
    uf = uI[S.dm.free]
    rhs = g.load(deg, f(g.quad_points(deg)))
    g.lift_dirichlet(uI, rhs)                          # F - K[:, fixed] u_I
    x = torch.zeros_like(rhs)
    x[:nvf] = torch.tensor(uf, device="cuda")
    x[nvf:] = torch.tensor(pex, device="cuda")
    r = (rhs - g.apply(x)).cpu().numpy()              # - K [u_I; p]
    scale = np.abs(rhs.cpu().numpy()).max()
    assert np.abs(r[:nvf]).max() <= 1e-11 * scale     # momentum rows
    assert np.abs(r[nvf:]).max() <= 1e-12 * scale     # divergence rows: B u_I = 0 elementwise

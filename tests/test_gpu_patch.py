"""The polynomial patch test on the GPU path, through the C ABI (convergence
theorem, Sec. 3: a solenoidal u in [P_k]^3 with p in P_{k-1} is reproduced
exactly): non-homogeneous Dirichlet data from vem_lift_dirichlet, the load
from vem_load, BDDC-PCG to rtol 1e-11.  The discrete velocity must equal
the interpolant of u (the oracle's DOFs of u) to 1e-10 and the pressure the
exact one up to its mean; the discrete velocity is divergence-free element
by element."""
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


@pytest.mark.parametrize("n,k,parts", [(4, 2, (2, 2, 2)), (3, 3, (3, 1, 1))])
def test_patch_test_on_the_gpu(pkg, n, k, parts):
    import torch
    from synth.mesh import box_partition
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
    pz = lambda p: p - (S.wmean @ p) / S.wmean.sum()
    g = pkg.VemSystem(mesh, k, nu)
    deg = 2 * k + 2
    rhs = g.load(deg, f(g.quad_points(deg)))
    g.lift_dirichlet(uI, rhs)
    bd = pkg.Bddc(g, box_partition(mesh, parts))
    x = torch.zeros_like(rhs)
    res = bd.solve(rhs, x, rtol=1e-11, maxit=300)
    assert res["status"] == 0
    x = x.cpu().numpy()
    nvf = g.n_vel_free
    uf = uI[S.dm.free]
    assert np.abs(x[:nvf] - uf).max() <= 1e-10 * np.abs(uf).max()
    assert np.abs(pz(x[nvf:]) - pz(pex)).max() <= 1e-8 * np.abs(pex).max()
    # elementwise divergence-free: the pressure rows of the residual
    r = (rhs - g.apply(torch.tensor(x, device="cuda"))).cpu().numpy()
    assert np.abs(r[nvf:]).max() <= 1e-10 * np.abs(rhs.cpu().numpy()).max()

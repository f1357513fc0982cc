"""Problem data: a manufactured divergence-free velocity and sinker fields.

Manufactured solution: psi = (x(1-x) y(1-y) z(1-z))^2 (1,1,1), u = curl psi,
p = 0.  With the form a(u,v) = int nu eps(u):eps(v) (no factor 2) and
div u = 0, the load is f = -div(nu eps(u)) = -(nu/2) Lap u for constant nu,
and Lap u = curl(Lap psi).

Multi-sinker data: nu(x) = nu_min + (nu_max - nu_min)(1 - chi(x)) with
chi(x) = prod_i (1 - exp(-delta max(0, |x - c_i| - omega/2)^2)), and the
buoyancy load f = (0, 0, -beta (1 - chi(x))).
"""
import numpy as np


def _g(t):
    return (t * (1 - t)) ** 2


def _g1(t):
    return 2 * t - 6 * t ** 2 + 4 * t ** 3


def _g2(t):
    return 2 - 12 * t + 12 * t ** 2


def _g3(t):
    return -12 + 24 * t


def manufactured_u(x):
    """u = curl psi at points x [..., 3]."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    px = _g1(X) * _g(Y) * _g(Z)
    py = _g(X) * _g1(Y) * _g(Z)
    pz = _g(X) * _g(Y) * _g1(Z)
    return np.stack([py - pz, pz - px, px - py], axis=-1)


def manufactured_f(x, nu=1.0):
    """f = -(nu/2) curl(Lap psi) at points x [..., 3]."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    gx, gy, gz = _g(X), _g(Y), _g(Z)
    g1x, g1y, g1z = _g1(X), _g1(Y), _g1(Z)
    g2x, g2y, g2z = _g2(X), _g2(Y), _g2(Z)
    g3x, g3y, g3z = _g3(X), _g3(Y), _g3(Z)
    # phi = Lap psi_s; its partial derivatives
    phx = g3x * gy * gz + g1x * g2y * gz + g1x * gy * g2z
    phy = g2x * g1y * gz + gx * g3y * gz + gx * g1y * g2z
    phz = g2x * gy * g1z + gx * g2y * g1z + gx * gy * g3z
    lap_u = np.stack([phy - phz, phz - phx, phx - phy], axis=-1)
    return -0.5 * nu * lap_u


def sinker_centres(n_sinkers, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n_sinkers, 3))


def _chi(x, centres, omega, delta):
    chi = np.ones(x.shape[:-1])
    for c in centres:
        d = np.maximum(0.0, np.linalg.norm(x - c, axis=-1) - 0.5 * omega)
        chi = chi * (1.0 - np.exp(-delta * d * d))
    return chi


def sinker_viscosity(x, centres, nu_min=1.0, nu_max=1e4, omega=0.1, delta=200.0):
    return nu_min + (nu_max - nu_min) * (1.0 - _chi(x, centres, omega, delta))


def sinker_load(x, centres, beta=10.0, omega=0.1, delta=200.0):
    f = np.zeros(x.shape)
    f[..., 2] = -beta * (1.0 - _chi(x, centres, omega, delta))
    return f

"""Pins of the uniform-grid oracle against closed-form flows: Couette (exact),
pressure-driven Poiseuille (parabola, second-order), Taylor-Green decay
(exp(-2 nu k^2 t), second-order), and a cavity at rest."""
import numpy as np
import pytest

from oracle.lattice import CS2, equilibrium, moments
from oracle.uniform import UniformLBM

NS, MV, OUT, PER = "noslip", "moving", "outlet", "periodic"
Z3 = (0.0, 0.0, 0.0)


def couette(dim, q, H, U, tau, steps):
    shape = (4, H) if dim == 2 else (4, H, 4)
    faces = [(PER, Z3), (PER, Z3), (NS, Z3), (MV, (U, 0.0, 0.0))]
    if dim == 3:
        faces += [(PER, Z3), (PER, Z3)]
    lbm = UniformLBM(dim, q, shape, tau, faces)
    for _ in range(steps):
        lbm.step()
    rho, u = lbm.moments()
    return u


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 27)])
def test_couette_exact(dim, q):
    H, U = 8, 0.05
    u = couette(dim, q, H, U, tau=0.8, steps=3000)
    y = np.arange(H) + 0.5
    ux = u[..., 0]
    prof = ux[0] if dim == 2 else ux[0, :, 0]
    assert np.max(np.abs(prof - U * y / H)) < 1e-12
    assert np.max(np.abs(u[..., 1])) < 1e-13


def test_couette_detects_wrong_wall_sign():
    # a moving wall with the wrong sign of the momentum term would drive -U
    u = couette(2, 9, 8, 0.05, 0.8, 3000)
    assert u[0, -1, 0] > 0


def poiseuille_error(H, tau=0.8, drho=1e-3):
    L = 4 * H
    faces = [(OUT, Z3, 1.0 + drho), (OUT, Z3, 1.0), (NS, Z3), (NS, Z3)]
    lbm = UniformLBM(2, 9, (L, H), tau, faces)
    nu = CS2 * (tau - 0.5)
    steps = int(3 * H * H / nu)
    for _ in range(steps):
        lbm.step()
    _, u = lbm.moments()
    prof = u[L // 2, :, 0]
    y = np.arange(H) + 0.5
    shape = y * (H - y)
    a = np.dot(prof, shape) / np.dot(shape, shape)      # one-parameter fit
    return np.max(np.abs(prof - a * shape)) / np.max(np.abs(prof)), prof


def test_poiseuille_parabola_second_order():
    e8, _ = poiseuille_error(8)
    e16, prof = poiseuille_error(16)
    assert prof.min() > 0                       # flows from high to low density
    assert e16 < 4e-3
    assert 2.5 < e8 / e16 < 6.0                 # ~4 for second order


def taylor_green_error(N, tau=0.8, U=0.01):
    k = 2 * np.pi / N
    faces = [(PER, Z3)] * 4
    lbm = UniformLBM(2, 9, (N, N), tau, faces)
    x = np.arange(N) + 0.5
    X, Y = np.meshgrid(x, x, indexing="ij")
    ux = -U * np.cos(k * X) * np.sin(k * Y)
    uy = U * np.sin(k * X) * np.cos(k * Y)
    p = -0.25 * U * U * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho = 1.0 + p / CS2
    u0 = np.stack([ux, uy], -1)
    lbm.f = equilibrium(lbm.vs, rho, u0)
    nu = CS2 * (tau - 0.5)
    t = int(round(1.0 / (2 * nu * k * k)))
    for _ in range(t):
        lbm.step()
    _, u = lbm.moments()
    amp = np.sum(u * u0) / np.sum(u0 * u0)
    return abs(amp / np.exp(-2 * nu * k * k * t) - 1.0)


def test_taylor_green_decay():
    e32 = taylor_green_error(32)
    e64 = taylor_green_error(64)
    assert e64 < 1e-2
    assert 2.5 < e32 / e64 < 6.0


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 27)])
def test_cavity_at_rest_stays_at_rest(dim, q):
    shape = (8, 8) if dim == 2 else (8, 8, 8)
    faces = [(NS, Z3)] * (2 * dim)
    faces[-1] = (MV, Z3)
    lbm = UniformLBM(dim, q, shape, 0.7, faces)
    f0 = lbm.f.copy()
    for _ in range(20):
        lbm.step()
    # rounding of the moment sums only (no momentum source anywhere)
    assert np.max(np.abs(lbm.f - f0)) < 1e-15

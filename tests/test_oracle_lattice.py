"""Pins of oracle.lattice against the paper's velocity-set figure and the exact
moment identities of the velocity sets and of the BGK equilibrium."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.lattice import (CS2, VelocitySet, bgk_collide, equilibrium, moments,
                            tau_level, velocities, weights_exact)

SETS = [(2, 9), (3, 19), (3, 27)]


def test_numbering_matches_figure(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "velocity_sets.txt"))
            if l.strip() and not l.startswith("#")]
    d2 = {int(r[1]): tuple(int(x) for x in r[2:]) for r in rows if r[0] == "D2Q9"}
    d3 = {int(r[1]): tuple(int(x) for x in r[2:]) for r in rows if r[0] == "D3Q27"}
    assert [tuple(v) for v in velocities(2, 9)] == [d2[i] for i in range(9)]
    assert [tuple(v) for v in velocities(3, 27)] == [d3[i] for i in range(27)]
    # D3Q19 is the first 19 directions of D3Q27
    assert [tuple(v) for v in velocities(3, 19)] == [d3[i] for i in range(19)]


def test_opposite_pairs_3d():
    for q in (19, 27):
        vs = VelocitySet(3, q)
        for k in range(1, q, 2):
            assert vs.opp[k] == k + 1 and vs.opp[k + 1] == k


@pytest.mark.parametrize("dim,q", SETS)
def test_weight_moments_exact(dim, q):
    c = velocities(dim, q)
    w = weights_exact(dim, q)
    cs2 = Fraction(1, 3)
    assert sum(w) == 1
    for a in range(dim):
        assert sum(wi * int(ci[a]) for wi, ci in zip(w, c)) == 0
        for b in range(dim):
            m2 = sum(wi * int(ci[a]) * int(ci[b]) for wi, ci in zip(w, c))
            assert m2 == (cs2 if a == b else 0)
    # odd third moments vanish, fourth moment is isotropic
    for a, b, g in itertools.product(range(dim), repeat=3):
        assert sum(wi * int(ci[a]) * int(ci[b]) * int(ci[g]) for wi, ci in zip(w, c)) == 0
    for a, b, g, e in itertools.product(range(dim), repeat=4):
        m4 = sum(wi * int(ci[a]) * int(ci[b]) * int(ci[g]) * int(ci[e]) for wi, ci in zip(w, c))
        iso = cs2 * cs2 * ((a == b) * (g == e) + (a == g) * (b == e) + (a == e) * (b == g))
        assert m4 == iso


@pytest.mark.parametrize("dim,q", SETS)
def test_equilibrium_moments(dim, q):
    vs = VelocitySet(dim, q)
    g = np.random.default_rng(1)
    rho = 1 + 0.1 * g.random(50)
    u = 0.1 * (g.random((50, dim)) - 0.5)
    feq = equilibrium(vs, rho, u)
    assert np.allclose(feq.sum(-1), rho, rtol=0, atol=1e-14)
    assert np.allclose(feq @ vs.cf, rho[:, None] * u, rtol=0, atol=1e-14)
    pi = np.einsum("np,pa,pb->nab", feq, vs.cf, vs.cf)
    expect = rho[:, None, None] * (CS2 * np.eye(dim) + u[:, :, None] * u[:, None, :])
    assert np.allclose(pi, expect, rtol=0, atol=1e-14)


def test_equilibrium_sign_reading():
    # the printed signs (-(c.u)^2/(2cs^4) + u.u/(2cs^2)) break the second moment
    vs = VelocitySet(2, 9)
    rho, u = np.ones(1), np.array([[0.1, 0.05]])
    cu = u @ vs.cf.T
    usq = (u * u).sum(-1)[:, None]
    printed = vs.w * rho[:, None] * (1 + cu / CS2 - cu * cu / (2 * CS2 ** 2) + usq / (2 * CS2))
    pi = np.einsum("np,pa,pb->nab", printed, vs.cf, vs.cf)
    assert not np.allclose(pi[0], CS2 * np.eye(2) + np.outer(u[0], u[0]), atol=1e-6)


@pytest.mark.parametrize("dim,q", SETS)
def test_bgk_conserves_and_relaxes(dim, q):
    vs = VelocitySet(dim, q)
    g = np.random.default_rng(2)
    rho = 1 + 0.05 * g.random(20)
    u = 0.05 * (g.random((20, dim)) - 0.5)
    f = equilibrium(vs, rho, u) + 1e-3 * (g.random((20, q)) - 0.5)
    fs, r, uu = bgk_collide(vs, f, 1.0)
    r2, u2 = moments(vs, fs)
    assert np.allclose(r2, r, atol=1e-14) and np.allclose(u2, uu, atol=1e-14)
    # omega = 1 relaxes fully onto the equilibrium
    assert np.allclose(fs, equilibrium(vs, r, uu), atol=1e-15)
    fs0, _, _ = bgk_collide(vs, f, 0.0)
    assert np.array_equal(fs0, f)


def test_tau_level_viscosity():
    # nu_L in level lattice units = cs^2 (tau_L - 1/2); physical nu = nu_L dx_L^2/dt_L
    # must be level independent with dx_L = dt_L = 2^-L
    nu0 = 0.0032
    for L in range(5):
        nu_L = CS2 * (tau_level(nu0, L) - 0.5)
        assert abs(nu_L * 2.0 ** (-L) - nu0) < 1e-15

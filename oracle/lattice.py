"""Velocity sets, BGK equilibrium and moments -- Section 2 (BGK, equilibrium and
moment equations; velocity-set figure).  Test infrastructure only.

Direction numbering follows the labels of the paper's velocity-set figure:

* D2Q9: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-).
* D3Q19/D3Q27: 0 rest, then opposite pairs (2k-1, 2k): 1/2 +-x, 3/4 +-y,
  5/6 +-z, 7/8 +-(x+y), 9/10 +-(x+z), 11/12 +-(y+z), 13/14 +-(x-y),
  15/16 +-(x-z), 17/18 +-(y-z), 19/20 +-(1,1,1), 21/22 +-(1,1,-1),
  23/24 +-(1,-1,1), 25/26 +-(-1,1,1).

The paper does not print the weights (it cites the standard textbook); the
standard Gauss-Hermite weights are used: they are the unique weights by speed
shell that satisfy the moment identities pinned in the tests.

Equilibrium: the paper's printed equilibrium has the signs of its last two
terms exchanged.  The reading used is the standard second-order form
    f_eq = w rho (1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)),
the only sign choice whose moments give rho, rho u and rho cs^2 I + rho u u.
"""
from fractions import Fraction

import numpy as np

CS2 = 1.0 / 3.0

D2Q9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]

D3Q19 = [(0, 0, 0),
         (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, -1, -1),
         (1, -1, 0), (-1, 1, 0), (1, 0, -1), (-1, 0, 1), (0, 1, -1), (0, -1, 1)]

D3Q27 = D3Q19 + [(1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
                 (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]

_SETS = {(2, 9): D2Q9, (3, 19): D3Q19, (3, 27): D3Q27}

# Standard weights by squared speed |c|^2 (textbook values, exact rationals).
_WEIGHTS = {
    (2, 9): {0: Fraction(4, 9), 1: Fraction(1, 9), 2: Fraction(1, 36)},
    (3, 19): {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)},
    (3, 27): {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)},
}


def velocities(dim, q):
    """Integer lattice vectors c_p, shape [Q, dim], in the paper's numbering."""
    return np.array(_SETS[(dim, q)], dtype=np.int64)


def weights_exact(dim, q):
    """Weights w_p as exact fractions (list of length Q)."""
    table = _WEIGHTS[(dim, q)]
    return [table[sum(x * x for x in c)] for c in _SETS[(dim, q)]]


def weights(dim, q):
    return np.array([float(w) for w in weights_exact(dim, q)], dtype=np.float64)


def opposite(dim, q):
    """Index of -c_p for every p."""
    c = velocities(dim, q)
    idx = {tuple(v): i for i, v in enumerate(c)}
    return np.array([idx[tuple(-v)] for v in c], dtype=np.int64)


class VelocitySet:
    def __init__(self, dim, q):
        self.dim, self.q = dim, q
        self.c = velocities(dim, q)
        self.cf = self.c.astype(np.float64)
        self.w = weights(dim, q)
        self.opp = opposite(dim, q)


def equilibrium(vs, rho, u):
    """Second-order BGK equilibrium (Section 2).  rho [...], u [..., dim] ->
    f_eq [..., Q]."""
    cu = u @ vs.cf.T                       # [..., Q]
    usq = np.sum(u * u, axis=-1)[..., None]
    return vs.w * rho[..., None] * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2)
                                    - usq / (2.0 * CS2))


def moments(vs, f):
    """rho = sum_p f_p, u = sum_p f_p c_p / rho (Section 2).  f [..., Q]."""
    rho = np.sum(f, axis=-1)
    u = (f @ vs.cf) / rho[..., None]
    return rho, u


def bgk_collide(vs, f, omega):
    """Post-collision f* = f - omega (f - f_eq(rho(f), u(f))) with
    omega = dt/tau (Section 4.3).  Returns (f*, rho, u)."""
    rho, u = moments(vs, f)
    feq = equilibrium(vs, rho, u)
    return f - omega * (f - feq), rho, u


def tau_level(nu0, level):
    """Relaxation time on level L (Section 4.3): nu = cs^2 (tau - dt/2) with
    dt_L = dt/2^L and dx_L = dt_L, so in level-L lattice units
    tau_L = 1/2 + 2^L (tau_0 - 1/2), tau_0 = nu0/cs^2 + 1/2 (nu0 in root
    lattice units)."""
    tau0 = nu0 / CS2 + 0.5
    return 0.5 + (2.0 ** level) * (tau0 - 0.5)

"""Pins of the oracle's refinement criterion (Section 4.4, Algorithm 3).

* The block vorticity in 3D (and 2D) against closed forms: for a velocity
  field linear in position, u = A x, the block-local first differences are
  exact and the curl is the constant vector (A_zy - A_yz, A_xz - A_zx,
  A_yx - A_xy); a rigid rotation u = Omega x r has curl 2 Omega; a symmetric
  A has no curl.  A transposed reshape, a swapped axis or a sign slip in a
  curl component changes |w|^2 for a generic A.
* Algorithm 3's thresholds: eps < T evaluated as |w|^2 < 4^T, strict.
* The mark rule on hand-set block maxima: a leaf is marked for refinement
  when L_des > L, a REFINED block (every child a leaf) for coarsening when
  L_des <= L, and a REFINED_WITH_CHILD block is never marked.
"""
import numpy as np
import pytest

import workloads as W
from oracle.forest import REFINED, REFINED_WITH_CHILD, UNREFINED
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM


def _set_linear_field(lbm, b, A):
    """Populations of block b at equilibrium with rho = 1 and u = A x, x the
    physical cell centre (u in lattice units = physical units, dx = dt)."""
    h = lbm.mesh.width(int(lbm.mesh.level[b])) / 4.0     # cell width, root-cell units
    x_cells = lbm.mesh.X[b] + (lbm.lc + 0.5) * h
    x_phys = x_cells * (lbm.cfg["length_x"] / lbm.cfg["nx"])
    u = x_phys @ np.asarray(A, np.float64).T
    lbm.f[b] = equilibrium(lbm.vs, np.ones(lbm.m), u)
    return u


def _curl_sq(A):
    A = np.asarray(A, np.float64)
    w = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    return float(w @ w)


def _rotation(omega):
    """Matrix of u = omega x r."""
    ox, oy, oz = omega
    return np.array([[0.0, -oz, oy], [oz, 0.0, -ox], [-oy, ox, 0.0]])


CENTRAL = [21, 22, 25, 26, 37, 38, 41, 42]               # roots (1..2, 1..2, 1..2)


def _three_level_3d():
    # the 2x2x2 central roots of a 4x4x4 root grid refined once
    cfg = W.cavity(dim=3, q=19, n=16, max_levels=4, max_blocks=64 + 8 * 24)
    lbm = ForestLBM(cfg)
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[CENTRAL] = 1
    lbm.mesh.adapt(m)
    assert all(lbm.mesh.status[r] == REFINED for r in CENTRAL)
    return lbm


@pytest.mark.parametrize("level", [0, 1])
def test_vorticity_3d_closed_forms(level):
    lbm = _three_level_3d()
    if level == 0:
        b = 43                                           # root (3, 2, 2)
    else:
        b = int(lbm.mesh.child0[21]) + 5                 # child (1, 0, 1) of root 21
    assert int(lbm.mesh.level[b]) == level
    rng = np.random.default_rng(11)
    cases = []
    for axis in range(3):                                # rigid rotation about each axis
        om = np.zeros(3)
        om[axis] = 0.03 * (axis + 1)
        cases.append((_rotation(om), 4.0 * float(om @ om)))
    om = np.array([0.021, -0.034, 0.017])
    cases.append((_rotation(om), 4.0 * float(om @ om)))
    S = rng.uniform(-0.05, 0.05, (3, 3))
    cases.append((S + S.T, 0.0))                         # pure strain: no curl
    for _ in range(4):                                   # generic gradients
        A = rng.uniform(-0.06, 0.06, (3, 3))
        cases.append((A, _curl_sq(A)))
    for A, expect in cases:
        u = _set_linear_field(lbm, b, A)
        assert np.max(np.abs(u)) < 0.2
        w2 = lbm.block_vorticity_sq(b)
        assert abs(w2 - expect) <= 1e-12 * max(1.0, expect) + 1e-14, (A, w2, expect)


def test_vorticity_3d_discriminates_axes():
    # a generic gradient whose |curl|^2 changes when the differences are taken
    # along permuted axes (a wrong [k][j][i] reshape: du_a/dx_b read as
    # du_a/dx_pi(b)), when component and derivative are exchanged in one
    # term, or when one difference enters with the wrong sign
    lbm = _three_level_3d()
    A = np.array([[0.01, 0.05, -0.02], [0.03, -0.01, 0.04], [-0.06, 0.02, 0.015]])
    _set_linear_field(lbm, 43, A)
    w2 = lbm.block_vorticity_sq(43)
    perms = [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0), (2, 0, 1)]
    others = [_curl_sq(A[:, list(p)]) for p in perms]
    for a in range(3):
        for c in range(a + 1, 3):
            B = A.copy()
            B[a, c], B[c, a] = A[c, a], A[a, c]
            others.append(_curl_sq(B) if _curl_sq(B) != _curl_sq(A) else np.inf)
    for a in range(3):
        for c in range(3):
            if a != c:
                B = A.copy()
                B[a, c] = -B[a, c]
                others.append(_curl_sq(B))
    assert abs(w2 - _curl_sq(A)) < 1e-14
    assert min(abs(w2 - o) for o in others) > 1e-5


def test_vorticity_2d_rotation():
    cfg = W.cavity(dim=2, q=9, n=16, max_levels=3)
    lbm = ForestLBM(cfg)
    for om in (0.02, -0.035):
        A = np.array([[0.004, -om], [om, -0.004]])       # rotation + strain
        dx = 1.0 / 16
        x = (lbm.lc + 0.5) * dx
        lbm.f[5] = equilibrium(lbm.vs, np.ones(16), (x + lbm.mesh.X[5] * dx) @ A.T)
        w2 = lbm.block_vorticity_sq(5)
        assert abs(w2 - 4 * om * om) < 1e-14


def test_desired_level_thresholds_are_strict():
    # L_max 4, N_start -2, N_inc 1: thresholds 4^-3, 4^-4, 4^-5 for p = 1, 2, 3
    lbm = _three_level_3d()
    cases = [(4.0 ** -3, 3), (np.nextafter(4.0 ** -3, 0), 2),
             (4.0 ** -4, 2), (np.nextafter(4.0 ** -4, 0), 1),
             (4.0 ** -5, 1), (np.nextafter(4.0 ** -5, 0), 0),
             (0.0, 0), (1e3, 3)]
    for w2, expect in cases:
        assert lbm.desired_level(w2) == expect, (w2, expect)


def test_criterion_mark_rule():
    lbm = _three_level_3d()
    mesh = lbm.mesh
    # refining child 7 of root 21 (all its level-1 neighbours exist) makes
    # root 21 REFINED_WITH_CHILD; root 42 stays REFINED (children leaves)
    m = np.zeros(mesh.cap, np.int8)
    m[int(mesh.child0[21]) + 7] = 1
    mesh.adapt(m)
    r21, r42 = 21, 42
    c21 = int(mesh.child0[r21])
    assert mesh.status[r21] == REFINED_WITH_CHILD
    assert mesh.status[r42] == REFINED
    assert mesh.status[c21 + 7] == REFINED
    assert mesh.status[c21 + 0] == UNREFINED and mesh.level[c21] == 1
    assert mesh.status[0] == UNREFINED and mesh.level[0] == 0
    t3, t4, t5 = 4.0 ** -3, 4.0 ** -4, 4.0 ** -5
    below = lambda t: float(np.nextafter(t, 0))
    w2 = {}
    for b in mesh.active_ids():
        w2[b] = 0.0                                      # L_des 0: no refinement
    expect = {}
    # leaves on level 0: refined when L_des > 0, i.e. w^2 >= 4^-5 (strict <)
    w2[0], expect[0] = t5, 1
    w2[1], expect[1] = below(t5), 0
    w2[2], expect[2] = 1.0, 1
    # leaves on level 1: refined when L_des >= 2, i.e. w^2 >= 4^-4
    w2[c21 + 1], expect[c21 + 1] = t4, 1
    w2[c21 + 2], expect[c21 + 2] = below(t4), 0
    # a leaf on the finest allowed level (L_max - 1 = 3 is not reached here;
    # a level-2 leaf with L_des 3 is marked, one with L_des 2 is not)
    c217 = int(mesh.child0[c21 + 7])
    w2[c217 + 0], expect[c217 + 0] = t3, 1
    w2[c217 + 1], expect[c217 + 1] = below(t3), 0
    # REFINED block on level 0 (children leaves): coarsened when L_des <= 0
    w2[r42], expect[r42] = below(t5), -1
    # REFINED block on level 1: coarsened when L_des <= 1 (L_des == L counts)
    w2[c21 + 7], expect[c21 + 7] = t5, -1
    # a REFINED_WITH_CHILD block is never marked, whatever its vorticity
    w2[r21], expect[r21] = 0.0, 0
    lbm.block_vorticity_sq = lambda b: w2[b]
    marks, got = lbm.criterion_marks()
    for b, e in expect.items():
        assert marks[b] == e, (b, marks[b], e)
    # every other leaf has L_des 0 = its level or less: unmarked; refined
    # blocks with L_des 0 above level 0 are coarsened
    for b in mesh.active_ids():
        if b in expect:
            continue
        st, L = mesh.status[b], mesh.level[b]
        want = -1 if st == REFINED else 0
        assert marks[b] == want, (b, st, L, marks[b])
    # a REFINED block on level 1 with L_des 2 > 1 keeps its children
    w2[c21 + 7] = t4
    marks, _ = lbm.criterion_marks()
    assert marks[c21 + 7] == 0

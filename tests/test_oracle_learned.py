"""Pins of oracle.learned: the MLP gradient against central finite differences,
and the block summaries on a linear velocity field (closed form)."""
import numpy as np

import workloads as W
from oracle import learned as LN
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    params = 0.3 * g.standard_normal(LN.NP)
    x = g.standard_normal((7, LN.IN))
    y = (g.random(7) < 0.4).astype(float)
    loss, grad = LN.loss_and_grad(params, x, y, pos_weight=2.5)
    z, p = LN.forward(params, x)
    assert np.isclose(loss, np.sum(-(2.5 * y * np.log(p) + (1 - y) * np.log(1 - p))))
    idx = g.choice(LN.NP, 60, replace=False)
    idx[0] = LN.NP - 1                        # b3
    h = 1e-6
    for i in idx:
        e = np.zeros(LN.NP)
        e[i] = h
        num = (LN.loss_and_grad(params + e, x, y, 2.5)[0]
               - LN.loss_and_grad(params - e, x, y, 2.5)[0]) / (2 * h)
        assert abs(num - grad[i]) <= 1e-6 * max(1.0, abs(num)), i


def test_block_features_linear_field():
    cfg = W.periodic_box(dim=3, q=19, n=8, nu0=0.01, max_levels=2)
    lbm = ForestLBM(cfg)
    b = 3
    dx = cfg["length_x"] / cfg["nx"]
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.6]])   # du_a/dx_b (physical)
    c = np.array([0.01, -0.02, 0.015])
    xc = lbm.lc * dx                          # cell positions within the block (physical)
    u = c + xc @ A.T
    lbm.f[b] = equilibrium(lbm.vs, np.ones(64), u)
    feat = LN.block_features(lbm, b)
    from oracle.lattice import moments
    _, um = moments(lbm.vs, lbm.f[b])
    assert np.allclose(um, u, atol=1e-15)
    assert np.allclose(feat[0:9], LN.squash(A.ravel()), atol=1e-9)
    assert np.allclose(feat[9:18], LN.squash(np.abs(A.ravel())), atol=1e-9)
    w = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    assert np.isclose(feat[24], LN.squash(np.linalg.norm(w)), atol=1e-9)
    assert np.isclose(feat[25], LN.squash(np.linalg.norm(w)), atol=1e-9)
    assert np.allclose(feat[20:23], 20 * u.mean(0), atol=1e-12)
    assert abs(feat[18]) < 1e-10 and abs(feat[19]) < 1e-10
    assert feat[26] == 0.0

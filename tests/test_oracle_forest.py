"""Pins of the block-forest oracle (oracle.forest, oracle.solver):

* with no refinement the forest equals the dense uniform-grid solver;
* mesh invariants after seeded random refine/coarsen sequences, checked by
  brute force (tiling, 2:1 balance, ID/gap partition, sibling contiguity,
  ID-set membership, cell classes by rasterisation);
* a worked example of the gap-stack allocation order;
* linear interpolation exact on multilinear data, equilibrium preserved,
  averaging of constants, average(interpolate(affine)) = affine;
* a static two-level Couette flow stays linear (pins the rescaling factor);
* Taylor-Green decay on a static two-level periodic forest;
* the vorticity criterion on a linear shear (closed form);
* the MLUPS update count against a brute-force leaf count;
* the momentum-exchange force against the fluid's momentum balance;
* every mark pattern on tiny forests (2x2 roots in 2D, 2x1x1 in 3D) over two
  calls: decisions from geometry alone, gap-stack group heads, invariants.
"""
import copy
import itertools

import numpy as np
import pytest

import workloads as W
from oracle.forest import (BLOCK_EDGE, GHOST, INACTIVE, INTERFACE, INTERIOR, NONE,
                           REFINED, REFINED_ANY, REFINED_PERMANENT, UNREFINED, Forest,
                           local_coords)
from oracle.lattice import CS2, equilibrium, moments
from oracle.solver import ForestLBM
from oracle.uniform import UniformLBM


# ------------------------------------------------------------------ helpers
def global_index(lbm, b):
    """Global cell indices (tuple of arrays) of the cells of root block b."""
    pos = (lbm.mesh.X[b][None, :] + lbm.lc).astype(np.int64)
    return tuple(pos[:, a] for a in range(lbm.dim))


def load_uniform(lbm, field):
    for b in range(lbm.mesh.n_root):
        lbm.f[b] = field[global_index(lbm, b)]


def to_uniform(lbm, shape, q):
    out = np.zeros(tuple(shape) + (q,))
    for b in range(lbm.mesh.n_root):
        out[global_index(lbm, b)] = lbm.f[b]
    return out


def random_state(vs, shape, seed):
    n = int(np.prod(shape))
    rho, u = W.random_macro(seed, n, vs.dim)
    f = equilibrium(vs, rho, u) + W.random_noise(seed + 1, (n, vs.q), 1e-3)
    return f.reshape(tuple(shape) + (vs.q,))


# ------------------------------------------------- forest == uniform grid
CASES = [
    ("cavity2d", lambda: W.cavity(dim=2, q=9, n=16, ny=12, max_levels=1)),
    ("cavity3d_q19", lambda: W.cavity(dim=3, q=19, n=8, ny=12, nz=8, max_levels=1)),
    ("periodic3d_q27", lambda: W.periodic_box(dim=3, q=27, n=8, ny=4, nz=12)),
    ("cylinder_small", lambda: W.channel_cylinder(q=19, nx=24, ny=16, nz=4, side=4,
                                                   cx=8, cy=8, max_levels=1)),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_forest_equals_uniform_single_level(name, mk):
    cfg = mk()
    lbm = ForestLBM(cfg)
    shape = [cfg["nx"], cfg["ny"], cfg["nz"]][:cfg["dim"]]
    uni = UniformLBM(cfg["dim"], cfg["q"], shape, lbm.tau[0], cfg["faces"])
    if cfg["solid"] is not None:
        uni.solid = to_uniform(lbm, shape, cfg["q"])[..., 0] * 0 != 0
        for b in range(lbm.mesh.n_root):
            uni.solid[global_index(lbm, b)] = lbm.solid[b]
    f0 = random_state(uni.vs, shape, 11)
    if cfg["solid"] is not None:
        f0[uni.solid] = lbm.rest
    uni.f = f0.copy()
    load_uniform(lbm, f0)
    for _ in range(6):
        uni.step()
        lbm.step()
    got = to_uniform(lbm, shape, cfg["q"])
    assert np.max(np.abs(got - uni.f)) <= 1e-15


# ------------------------------------------------------ mesh invariants
def brute_force_check(mesh: Forest):
    d, nc = mesh.dim, mesh.nc
    act = mesh.active_ids()
    aset = set(act)
    # ID sets hold exactly the active blocks of each level, no duplicates
    assert len(act) == len(aset)
    for L, ids in enumerate(mesh.id_sets):
        assert all(mesh.level[b] == L for b in ids)
    # gap set and active IDs partition the capacity
    gaps = set(mesh.gap)
    assert len(gaps) == len(mesh.gap)
    assert gaps.isdisjoint(aset)
    assert gaps | aset == set(range(mesh.cap))
    assert all(mesh.status[b] == INACTIVE for b in gaps)
    # children are contiguous and point back to their parent
    for b in act:
        if mesh.status[b] in REFINED_ANY:
            c0 = mesh.child0[b]
            for c in range(nc):
                ch = c0 + c
                assert ch in aset and mesh.parent[ch] == b
                off = np.array([(c >> a) & 1 for a in range(d)])
                w = mesh.width(mesh.level[ch])
                assert np.array_equal(mesh.X[ch], mesh.X[b] + off * w)
        else:
            assert mesh.status[b] == UNREFINED and mesh.child0[b] == NONE
    # leaves tile the domain exactly once (rasterised on the finest grid)
    fine = 2 ** (mesh.lmax - 1)
    cover = np.zeros(tuple(int(e) * fine for e in mesh.extent), np.int64)
    level_of = np.full(cover.shape, -1)
    for b in act:
        if mesh.status[b] != UNREFINED:
            continue
        lo = (mesh.X[b] * fine).astype(np.int64)
        n = int(mesh.width(mesh.level[b]) * fine)
        sl = tuple(slice(lo[a], lo[a] + n) for a in range(d))
        cover[sl] += 1
        level_of[sl] = mesh.level[b]
    assert np.all(cover == 1)
    # 2:1 balance over the full neighbourhood (incl. periodic wrap)
    for a in range(d):
        for shift in (-1, 1):
            other = np.roll(level_of, shift, axis=a)
            diff = np.abs(level_of - other)
            if mesh.faces[2 * a][0] != "periodic":
                idx = [slice(None)] * d
                idx[a] = 0 if shift == 1 else -1
                diff[tuple(idx)] = 0
            assert diff.max() <= 1
    # diagonal balance: every leaf's 3^d neighbourhood of finest cells
    for sh in itertools.product((-1, 0, 1), repeat=d):
        other = level_of
        valid = np.ones(cover.shape, bool)
        for a, s in enumerate(sh):
            if s == 0:
                continue
            other = np.roll(other, s, axis=a)
            if mesh.faces[2 * a][0] != "periodic":
                idx = [slice(None)] * d
                idx[a] = 0 if s == 1 else -1
                valid[tuple(idx)] = False
        assert np.abs(level_of - other)[valid].max() <= 1


def brute_force_classes(mesh: Forest, b):
    """Cell classes of block b from a rasterisation of same-level coverage."""
    d = mesh.dim
    L = mesh.level[b]
    n_l = np.array([int(e) * 2 ** L for e in mesh.extent])
    covered = np.zeros(n_l, bool)
    for o in mesh.id_sets[L]:
        lo = (mesh.X[o] * 2 ** L).astype(np.int64)
        covered[tuple(slice(lo[a], lo[a] + 4) for a in range(d))] = True
    pos = (mesh.X[b] * 2 ** L).astype(np.int64)[None, :] + local_coords(d)
    best = np.full(len(pos), 99)
    for off in itertools.product(range(-4, 5), repeat=d):
        y = pos + np.array(off)
        ok = np.ones(len(pos), bool)
        for a in range(d):
            out = (y[:, a] < 0) | (y[:, a] >= n_l[a])
            if mesh.faces[2 * a][0] == "periodic":
                y[:, a] %= n_l[a]
            else:
                ok &= ~out
                y[:, a] = np.clip(y[:, a], 0, n_l[a] - 1)
        unc = ok & ~covered[tuple(y[:, a] for a in range(d))]
        best = np.where(unc, np.minimum(best, max(abs(o) for o in off)), best)
    return np.where(best <= 2, GHOST, np.where(best <= 4, INTERFACE, INTERIOR))


def geometric_nbr(mesh: Forest, b):
    """Neighbour IDs of block b by scanning every active block's box."""
    d = mesh.dim
    w = mesh.width(mesh.level[b])
    out = []
    for k in range(mesh.nk):
        pos = mesh.X[b] + mesh.dirs[k] * w
        wall = False
        for a in range(d):
            if pos[a] < 0 or pos[a] >= mesh.extent[a]:
                if mesh.faces[2 * a][0] == "periodic":
                    pos[a] %= mesh.extent[a]
                else:
                    wall = True
        if wall:
            out.append("wall")
            continue
        hit = [o for o in mesh.active_ids() if mesh.level[o] == mesh.level[b]
               and np.array_equal(mesh.X[o], pos)]
        assert len(hit) <= 1
        out.append(hit[0] if hit else NONE)
    return out


def with_roots(cfg, ids):
    cfg = dict(cfg)
    cfg["root_ids"] = ids(cfg)
    return cfg


MESHES = [
    ("2d_cavity_3x3", lambda: W.cavity(dim=2, n=12, max_levels=4, max_blocks=9 * 40)),
    ("2d_periodic_2x3", lambda: W.periodic_box(dim=2, n=8, ny=12, max_levels=3, max_blocks=200)),
    ("3d_cavity_2x2x2", lambda: W.cavity(dim=3, n=8, max_levels=3, max_blocks=8 * 30)),
    ("2d_cavity_4x3_shuffled", lambda: with_roots(
        W.cavity(dim=2, n=16, ny=12, max_levels=3, max_blocks=12 * 20),
        lambda c: W.shuffled_root_ids(c, 5))),
    ("3d_periodic_3x2x2_morton", lambda: with_roots(
        W.periodic_box(dim=3, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 25),
        W.morton_root_ids)),
]


@pytest.mark.parametrize("name,mk", MESHES, ids=[m[0] for m in MESHES])
def test_random_adaptation_invariants(name, mk):
    cfg = mk()
    mesh = Forest(cfg)
    for it in range(12):
        marks = W.random_marks(100 + it, mesh.cap, 0.35, 0.35)
        res = mesh.adapt(marks)
        brute_force_check(mesh)
        for b in mesh.active_ids()[:: max(1, len(mesh.active_ids()) // 12)]:
            geo = geometric_nbr(mesh, b)
            for k, g in enumerate(geo):
                if g == "wall":
                    assert mesh.nbr[b, k] <= -2
                else:
                    assert mesh.nbr[b, k] == g
            assert np.array_equal(mesh.cell_classes(b), brute_force_classes(mesh, b))


def test_capacity_cancels_refinement():
    cfg = W.cavity(dim=2, n=8, max_levels=3, max_blocks=4 + 4)   # room for one group
    mesh = Forest(cfg)
    marks = np.zeros(mesh.cap, np.int8)
    marks[[0, 1]] = 1
    res = mesh.adapt(marks)
    assert res["capacity_error"] and res["n_refined"] == 0
    assert mesh.counts() == [4, 0, 0]
    marks[1] = 0
    res = mesh.adapt(marks)
    assert not res["capacity_error"] and mesh.child0[0] == 4


def test_allocation_order_worked_example():
    # 2x2 root blocks (IDs 0..3), capacity 4 + 4 groups of 4.
    cfg = W.cavity(dim=2, n=8, max_levels=3, max_blocks=20)
    mesh = Forest(cfg)
    assert mesh.gap[-1] == 4 and mesh.gap[0] == 19      # reverse enumeration
    m = np.zeros(mesh.cap, np.int8)
    m[[2, 1]] = 1                      # ascending ID order decides: 1 then 2
    mesh.adapt(m)
    assert mesh.child0[1] == 4 and mesh.child0[2] == 8
    assert mesh.id_sets[1] == [4, 5, 6, 7, 8, 9, 10, 11]
    m[:] = 0
    m[1] = -1                          # coarsen block 1: frees 4..7
    mesh.adapt(m)
    assert mesh.id_sets[1] == [8, 9, 10, 11]
    assert mesh.gap[-4:] == [7, 6, 5, 4]
    m[:] = 0
    m[[0, 3]] = 1                      # block 0 takes the freed group 4..7
    mesh.adapt(m)
    assert mesh.child0[0] == 4 and mesh.child0[3] == 12
    assert mesh.id_sets[1] == [8, 9, 10, 11, 4, 5, 6, 7, 12, 13, 14, 15]
    assert mesh.status[[0, 1, 2, 3]].tolist() == [REFINED, UNREFINED, REFINED, REFINED]


def test_coarsen_reverted_next_to_finer_blocks():
    cfg = W.cavity(dim=2, n=8, max_levels=4, max_blocks=4 + 4 * 8)
    mesh = Forest(cfg)
    m = np.zeros(mesh.cap, np.int8)
    m[[0, 1, 2, 3]] = 1
    mesh.adapt(m)                           # all four roots refined
    child_of_1 = mesh.child0[1]
    # refine the child of block 0 that touches block 1 (child c = 1: +x side)
    m[:] = 0
    m[mesh.child0[0] + 1] = 1
    mesh.adapt(m)
    # coarsening block 1 would put level 0 next to level 2: reverted
    m[:] = 0
    m[1] = -1
    res = mesh.adapt(m)
    assert res["n_coarsened"] == 0 and mesh.child0[1] == child_of_1
    # blocks 2 and 3 do not touch the level-2 region [2,4]x[0,2]: allowed
    m[:] = 0
    m[[2, 3]] = -1
    assert mesh.adapt(m)["n_coarsened"] == 2
    brute_force_check(mesh)
    # block 0 cannot be coarsened: it has a refined child
    m[:] = 0
    m[0] = -1
    assert mesh.adapt(m)["n_coarsened"] == 0


# ------------------------------------------ interpolation and averaging
def test_interpolation_exact_on_multilinear():
    for dim, q in ((2, 9), (3, 19)):
        lbm = ForestLBM(W.periodic_box(dim=dim, q=q, n=8, max_levels=2))
        Wt = lbm._interp_weights()
        x = -0.25 + 0.5 * lbm.lc
        corners = np.array([[(a >> ax) & 1 for ax in range(dim)] for a in range(2 ** dim)], float)
        for mono in itertools.product((0, 1), repeat=dim):
            Fc = np.prod(corners ** np.array(mono), axis=1)
            expect = np.prod(x ** np.array(mono), axis=1)
            assert np.allclose(Wt @ Fc, expect, atol=1e-15), mono


def two_level_lbm(cfg, refine_ids):
    lbm = ForestLBM(cfg)
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[refine_ids] = 1
    res = lbm.mesh.adapt(m)
    lbm.interpolate(res["new_children"], "all")
    return lbm


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19)])
def test_cubic_interpolation_exact_on_cubic_equilibria(dim, q):
    """Cubic interpolation (Section 3.4.2) reproduces every population of an
    equilibrium whose density and velocity are affine in space: f_eq(rho(x),
    u(x)) has degree <= 3 in each coordinate, and rescaling leaves an
    equilibrium unchanged.  Positions come from the forest geometry (cell
    centres of parent and children), not from the interpolation code; linear
    interpolation must miss the same data."""
    errs = {}
    for kind in ("cubic", "linear"):
        cfg = W.periodic_box(dim=dim, q=q, n=8, max_levels=2, max_blocks=None)
        cfg["interp"] = kind
        lbm = ForestLBM(cfg)
        g = np.random.default_rng(4)
        a_rho, b_rho = 1.0, 0.01 * g.standard_normal(dim)
        a_u, B_u = 0.02 * g.standard_normal(dim), 0.006 * g.standard_normal((dim, dim))

        def state(x):
            return equilibrium(lbm.vs, a_rho + x @ b_rho, a_u + x @ B_u.T)

        par = 0
        lbm.f[par] = state(lbm.cell_centres(par))
        m = np.zeros(lbm.mesh.cap, np.int8)
        m[par] = 1
        res = lbm.mesh.adapt(m)
        kids = res["new_children"]
        assert len(kids) == 2 ** dim
        lbm.interpolate(kids, "all")
        errs[kind] = max(np.abs(lbm.f[c] - state(lbm.cell_centres(c))).max() for c in kids)
    assert errs["cubic"] <= 1e-13, errs
    assert errs["linear"] >= 1e-7, errs


def test_cubic_weights_are_tensor_lagrange():
    """The Vandermonde-inverse weights equal the product of the 1D cubic
    Lagrange bases on the nodes 0, 1/3, 2/3, 1 (the unique interpolant in the
    tensor-product cubic space)."""
    lbm = ForestLBM(W.periodic_box(dim=3, q=19, n=8, max_levels=2))
    Ws = lbm._cubic_weights()
    nodes = np.array([0.0, 1.0, 2.0, 3.0]) / 3.0

    def lag(x, mnode):
        out = 1.0
        for j in range(4):
            if j != mnode:
                out *= (x - nodes[j]) / (nodes[mnode] - nodes[j])
        return out

    for c in (0, 5, 7):
        off = [(c >> ax) & 1 for ax in range(3)]
        for cell in (0, 21, 63):
            I = [cell % 4, (cell // 4) % 4, cell // 16]
            x = [-1 / 12 + I[a] / 6 + off[a] * 2 / 3 for a in range(3)]
            for U in (0, 17, 42, 63):
                mm = [U % 4, (U // 4) % 4, U // 16]
                want = lag(x[0], mm[0]) * lag(x[1], mm[1]) * lag(x[2], mm[2])
                assert abs(Ws[c][cell, U] - want) <= 1e-14, (c, cell, U)


def test_interpolation_preserves_equilibrium():
    cfg = W.periodic_box(dim=3, q=19, n=8, max_levels=2, nu0=0.02)
    lbm = ForestLBM(cfg)
    rho, u = 1.01, np.array([0.03, -0.01, 0.02])
    feq = equilibrium(lbm.vs, np.array([rho]), u[None])[0]
    lbm.f[:] = feq
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[0] = 1
    res = lbm.mesh.adapt(m)
    lbm.interpolate(res["new_children"], "all")
    for c in res["new_children"]:
        assert np.max(np.abs(lbm.f[c] - feq)) < 1e-15


def test_averaging_constant_and_inverse_of_interpolation():
    cfg = W.periodic_box(dim=2, q=9, n=8, max_levels=2, nu0=0.02)
    lbm = ForestLBM(cfg)
    g = np.random.default_rng(5)
    rho = 1 + 0.01 * g.random(16)
    u = 0.02 * (g.random((16, 2)) - 0.5)
    # parent block 0: affine rescaled field => after interpolation every
    # child cell holds the affine value; averaging recovers the parent cell
    x = lbm.lc.astype(float)
    rho = 1.0 + 0.01 * x[:, 0] - 0.02 * x[:, 1]
    u = np.stack([0.01 * x[:, 1], 0.003 * x[:, 0]], -1)
    feq = equilibrium(lbm.vs, rho, u)
    # non-equilibrium part affine too (rescaling is then affine as well)
    lbm.f[0] = feq
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[0] = 1
    res = lbm.mesh.adapt(m)
    lbm.interpolate(res["new_children"], "all")
    before = lbm.f[0].copy()
    lbm.f[0] = 0.0
    lbm.average(res["new_children"], "sync")
    # sync averaging writes the parent cells over non-ghost children only
    written = np.any(lbm.f[0] != 0.0, axis=1)
    assert written.sum() == 4
    # equilibrium is quadratic in u: recovered to second order only
    assert np.max(np.abs(lbm.f[0][written] - before[written])) < 2e-5
    # constants are reproduced exactly
    lbm.f[res["new_children"]] = lbm.rest
    lbm.average(res["new_children"], "sync")
    assert np.max(np.abs(lbm.f[0][written] - lbm.rest)) < 1e-16


def test_averaging_children_are_geometric():
    cfg = W.periodic_box(dim=3, q=19, n=8, max_levels=2)
    lbm = ForestLBM(cfg)
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[3] = 1
    res = lbm.mesh.adapt(m)
    par = 3
    pc = lbm.cell_centres(par)
    for ch in res["new_children"]:
        cc = lbm.cell_centres(ch)
        corners = lbm.quadrant_cells(ch - lbm.mesh.child0[par])
        for a in range(8):
            kids = []
            for s in range(8):
                o = [2 * ((a >> ax) & 1) + ((s >> ax) & 1) for ax in range(3)]
                kids.append(o[0] + 4 * o[1] + 16 * o[2])
            # the 8 children lie inside the parent cell and average to its centre
            h = 0.5
            assert np.all(np.abs(cc[kids] - pc[corners[a]]) <= h / 2 + 1e-12)
            assert np.allclose(cc[kids].mean(0), pc[corners[a]])


# ------------------------------------------------------- level stepping
def couette_two_level(ratio_scale=None, steps=2600, interp="linear"):
    cfg = W.cavity(dim=2, q=9, n=16, max_levels=2, max_blocks=16 + 8 * 4)
    cfg["interp"] = interp
    cfg["faces"] = [("periodic", (0, 0, 0)), ("periodic", (0, 0, 0)),
                    ("noslip", (0, 0, 0)), ("moving", (0.05, 0.0, 0.0))]
    cfg["nu0"] = 0.25
    lbm = ForestLBM(cfg)
    # refine the middle band y in [4, 12): root blocks with by = 1, 2
    ids = [b for b in range(16) if (b // 4) in (1, 2)]
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[ids] = 1
    res = lbm.mesh.adapt(m)
    assert lbm.mesh.counts() == [16, 32]
    lbm.interpolate(res["new_children"], "all")
    if ratio_scale is not None:
        lbm._rescaled_orig = lbm._rescaled
        lbm._rescaled = lambda f, ratio: lbm._rescaled_orig(f, ratio_scale)
    lbm.step(steps)
    lbm.sync()
    rho, u = lbm.macroscopic()
    err = 0.0
    for b in lbm.mesh.active_ids():
        if lbm.mesh.status[b] != UNREFINED:
            continue
        y = lbm.cell_centres(b)[:, 1]
        err = max(err, np.max(np.abs(u[b, :, 0] - 0.05 * y / 16.0)))
    return err


def test_two_level_couette_linear():
    # correct Dupuis-Chopard factors: the linear profile survives two levels
    assert couette_two_level(None) < 1e-10
    # without rescaling (factor 1) the interface visibly breaks it
    assert couette_two_level(1.0, steps=1000) > 1e-5


def test_two_level_couette_linear_cubic():
    # cubic interpolation reproduces the linear profile as well
    assert couette_two_level(None, interp="cubic") < 1e-10


@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_taylor_green_two_level(interp):
    N, tau_root = 32, 0.8
    nu0 = CS2 * (tau_root - 0.5)
    cfg = W.periodic_box(dim=2, q=9, n=N, nu0=nu0, max_levels=2, max_blocks=64 + 4 * 64)
    cfg["interp"] = interp
    lbm = ForestLBM(cfg)
    k = 2 * np.pi / N
    U = 0.01

    def field(x):
        ux = -U * np.cos(k * x[:, 0]) * np.sin(k * x[:, 1])
        uy = U * np.sin(k * x[:, 0]) * np.cos(k * x[:, 1])
        p = -0.25 * U * U * (np.cos(2 * k * x[:, 0]) + np.cos(2 * k * x[:, 1]))
        return 1 + p / CS2, np.stack([ux, uy], -1)

    m = np.zeros(lbm.mesh.cap, np.int8)
    m[[b for b in range(64) if 2 <= b % 8 <= 4 and 2 <= b // 8 <= 5]] = 1
    lbm.mesh.adapt(m)
    assert lbm.mesh.counts() == [64, 48]
    for b in lbm.mesh.active_ids():
        r, uu = field(lbm.cell_centres(b))
        lbm.f[b] = equilibrium(lbm.vs, r, uu)
    t = int(round(1.0 / (2 * nu0 * k * k)))
    lbm.step(t)
    lbm.sync()
    num = den = 0.0
    for b in lbm.mesh.active_ids():
        if lbm.mesh.status[b] != UNREFINED:
            continue
        wgt = (lbm.mesh.width(lbm.mesh.level[b]) / 4) ** 2
        _, u0 = field(lbm.cell_centres(b))
        _, u = moments(lbm.vs, lbm.f[b])
        num += wgt * np.sum(u * u0)
        den += wgt * np.sum(u0 * u0)
    amp = num / den
    assert abs(amp / np.exp(-2 * nu0 * k * k * t) - 1) < 2e-2


def test_refined_patch_static_flow_stays_static():
    # uniform flow through a periodic two-level forest is an exact solution
    cfg = W.periodic_box(dim=3, q=19, n=8, max_levels=2, nu0=0.01)
    lbm = ForestLBM(cfg)
    feq = equilibrium(lbm.vs, np.ones(1), np.array([[0.02, 0.01, -0.015]]))[0]
    lbm.f[:] = feq
    m = np.zeros(lbm.mesh.cap, np.int8)
    m[0] = 1
    res = lbm.mesh.adapt(m)
    lbm.interpolate(res["new_children"], "all")
    lbm.step(5)
    lbm.sync()
    for b in lbm.mesh.active_ids():
        assert np.max(np.abs(lbm.f[b] - feq)) < 1e-14


# ------------------------------------------------------------- criterion
def test_criterion_linear_shear():
    cfg = W.cavity(dim=2, q=9, n=16, max_levels=4)   # N_start -2, N_inc 1
    lbm = ForestLBM(cfg)
    dx = 1.0 / 16
    for s, expect in ((0.2, 3), (0.1, 2), (0.05, 1), (0.01, 0)):
        # u_x = s * y (physical), lattice u = s * dx * j per cell
        j = lbm.lc[:, 1].astype(float)
        u = np.stack([s * dx * j, np.zeros(16)], -1)
        lbm.f[0] = equilibrium(lbm.vs, np.ones(16), u)
        w2 = lbm.block_vorticity_sq(0)
        assert abs(w2 - s * s) < 1e-12
        # thresholds 2^-3, 2^-4, 2^-5 for p = 1, 2, 3
        assert lbm.desired_level(w2) == expect


def test_mlups_count_brute_force():
    cfg = W.cavity(dim=3, q=19, n=8, max_levels=3, max_blocks=8 * 20)
    lbm = ForestLBM(cfg)
    for it in range(4):
        lbm.mesh.adapt(W.random_marks(7 + it, lbm.mesh.cap, 0.5, 0.2))
    leaves = [b for b in lbm.mesh.active_ids() if lbm.mesh.status[b] == UNREFINED]
    brute = sum(2 ** lbm.mesh.level[b] * 64 for b in leaves)
    assert lbm.updates_per_coarse_step() == brute


# ---------------------------------------------------------- distance rule
def brute_distance(box_a, box_b, n=41):
    """Minimum Euclidean distance between two axis-aligned squares by dense
    sampling of both (exact to the sampling step)."""
    def pts(b):
        xs = np.linspace(b[0], b[1], n)
        ys = np.linspace(b[2], b[3], n)
        X, Y = np.meshgrid(xs, ys)
        return np.stack([X.ravel(), Y.ravel()], 1)
    pa, pb = pts(box_a), pts(box_b)
    d = np.sqrt(((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1))
    return d.min(), max((box_a[1] - box_a[0]), (box_b[1] - box_b[0])) / (n - 1)


def test_distance_rule_matches_brute_force():
    cfg = W.channel_cylinder(q=19, nx=48, ny=24, nz=4, side=4, cx=16, cy=12, max_levels=3,
                             refine_dist=0.15)
    lbm = ForestLBM(cfg)
    lbm.mesh.adapt(np.ones(lbm.mesh.cap, np.int8))      # two levels to test
    lbm.mesh.adapt(np.ones(lbm.mesh.cap, np.int8))
    x0, x1, y0, y1 = cfg["solid"]
    checked = 0
    for b in lbm.mesh.active_ids():
        L = int(lbm.mesh.level[b])
        w = lbm.mesh.width(L)
        X = lbm.mesh.X[b]
        thr = 0.15 * cfg["nx"] / 2 ** L
        d_solid, step = brute_distance((X[0], X[0] + w, X[1], X[1] + w), (x0, x1, y0, y1))
        d_out = cfg["nx"] - (X[0] + w)
        near = min(d_solid, d_out)
        if abs(near - thr) <= 2 * step:
            continue                                      # undecidable at this sampling
        assert lbm.within_refine_distance(b) == (near < thr), b
        checked += 1
    assert checked > 50


def test_frozen_blocks_are_never_coarsened():
    cfg = W.cavity(dim=2, n=8, max_levels=3, max_blocks=4 + 4 * 8)
    mesh = Forest(cfg)
    m = np.zeros(mesh.cap, np.int8)
    m[[0, 1]] = [2, 1]                                   # 0 frozen, 1 plain
    mesh.adapt(m)
    assert mesh.status[0] == 4 and mesh.status[1] == REFINED
    m[:] = 0
    m[[0, 1]] = -1
    res = mesh.adapt(m)
    assert res["n_coarsened"] == 1 and mesh.status[0] == 4 and mesh.status[1] == UNREFINED
    brute_force_check(mesh)


# ------------------------------------------------------- root numbering
def test_morton_root_ids_follow_the_z_curve():
    cfg = W.periodic_box(dim=3, n=16, max_levels=1)
    ids = W.morton_root_ids(cfg)
    assert sorted(ids.tolist()) == list(range(64))
    pos = W.root_positions(cfg)
    by_id = pos[np.argsort(ids)]                      # position of ID 0, 1, ...
    # each aligned group of 8 IDs is a 2x2x2 cube, each of 64 a 4x4x4 cube
    for g in range(8):
        cube = by_id[8 * g:8 * g + 8]
        assert np.all(cube.max(0) - cube.min(0) == 1)
    assert np.array_equal(by_id[:8].min(0), [0, 0, 0])
    assert np.array_equal(by_id[1], [1, 0, 0]) and np.array_equal(by_id[2], [0, 1, 0])
    assert np.array_equal(by_id[4], [0, 0, 1])


@pytest.mark.parametrize("dim", [2, 3])
def test_root_numbering_is_a_relabelling(dim):
    """Fields of a two-level forest with shuffled root IDs equal, position by
    position and bit for bit, those of the lexicographic numbering."""
    base = (W.cavity(dim=2, q=9, n=16, ny=12, max_levels=2, max_blocks=12 * 6) if dim == 2 else
            W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=2, max_blocks=12 * 10))
    runs, roots = [], []
    for ids in (None, W.shuffled_root_ids(base, 11)):
        cfg = dict(base)
        if ids is not None:
            cfg["root_ids"] = ids
        lbm = ForestLBM(cfg)
        m = np.zeros(cfg["max_blocks"], np.int8)
        for b in range(lbm.mesh.n_root):                  # refine by position
            if lbm.mesh.X[b][0] >= 4 and lbm.mesh.X[b][1] >= 4:
                m[b] = 1
        lbm.adapt(m)
        # the same state, a function of the cell position
        for b in lbm.mesh.active_ids():
            x = lbm.cell_centres(b)
            rho = 1.0 + 0.01 * np.sin(0.7 * x[:, 0]) * np.cos(0.4 * x[:, 1])
            u = 0.02 * np.stack([np.sin(0.3 * x[:, (a + 1) % dim] + a) for a in range(dim)], 1)
            lbm.f[b] = equilibrium(lbm.vs, rho, u)
        lbm.step(3)
        out = {}
        for b in lbm.mesh.active_ids():
            key = tuple(np.round(lbm.mesh.X[b] * 8).astype(np.int64)) + (int(lbm.mesh.level[b]),)
            out[key] = lbm.f[b].copy()
        runs.append(out)
        roots.append(lbm.mesh.X[:lbm.mesh.n_root].copy())
    assert not np.array_equal(roots[0], roots[1])          # the IDs did move
    assert runs[0].keys() == runs[1].keys() and len(runs[0]) > 0
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_wall_distance_rule_matches_brute_force():
    """Wall faces as distance targets: a leaf is within d_spec / 2^L of a wall
    exactly when the nearest of its sampled points is (brute force over the
    block's boundary points and the wall planes)."""
    cfg = W.cavity(dim=3, q=19, n=16, max_levels=3, max_blocks=64 * 20, refine_dist=0.1,
                   refine_dist_freeze=1)
    lbm = ForestLBM(cfg)
    lbm.mesh.adapt(np.ones(lbm.mesh.cap, np.int8))
    checked = within = 0
    n = cfg["nx"]
    for b in lbm.mesh.active_ids():
        L = int(lbm.mesh.level[b])
        w = lbm.mesh.width(L)
        X = lbm.mesh.X[b]
        thr = 0.1 * n / 2 ** L
        g = np.linspace(0.0, 1.0, 9)
        pts = X + w * np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        d = np.min(np.concatenate([pts, n - pts], axis=1))   # every face is a wall
        if abs(d - thr) < 1e-9:
            continue
        assert lbm.within_refine_distance(b) == (d < thr), b
        checked += 1
        within += d < thr
    assert checked > 100 and 0 < within < checked
    # the criterion freezes the blocks it refines by distance
    marks, _ = lbm.criterion_marks()
    leaves = [b for b in lbm.mesh.active_ids() if lbm.mesh.status[b] == UNREFINED]
    assert any(marks[b] == 2 for b in leaves)
    assert all(marks[b] in (1, 2) for b in leaves if lbm.within_refine_distance(b))


@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_pressure_continuous_across_interfaces(interp):
    """Section 5.3's observation that the pressure is continuous across
    coarse-fine interfaces: a pressure-driven channel (anti-bounce-back inlet
    and outlet at rho 1 +- 0.001, no-slip walls) with a refined band in the
    middle, run to steady state.  Along the centre line the density falls
    linearly; at both interfaces the step between the last coarse and the
    first fine cell deviates from that line by under 10 % of the drop over one
    coarse cell."""
    cfg = W.cavity(dim=2, q=9, n=32, ny=16, max_levels=2, max_blocks=32 + 8 * 4)
    cfg["faces"] = [("outlet", (0.0, 0.0, 0.0), 1.001), ("outlet", (0.0, 0.0, 0.0), 0.999),
                    ("noslip", (0.0, 0.0, 0.0)), ("noslip", (0.0, 0.0, 0.0))]
    cfg["nu0"] = 1.0 / 6.0
    cfg["interp"] = interp
    lbm = ForestLBM(cfg)
    m = np.zeros(lbm.mesh.cap, np.int8)
    for b in range(lbm.mesh.n_root):
        if lbm.mesh.X[b][0] in (12.0, 16.0):
            m[b] = 1
    lbm.adapt(m)
    assert lbm.mesh.counts() == [32, 32]
    lbm.step(3000)
    lbm.sync()
    xs, rs = [], []
    for b in lbm.mesh.active_ids():
        if lbm.mesh.status[b] != UNREFINED:
            continue
        c = lbm.cell_centres(b)
        rho, _ = moments(lbm.vs, lbm.f[b])
        sel = np.abs(c[:, 1] - 8.0) < 0.6
        xs += list(c[sel, 0])
        rs += list(rho[sel])
    xs, rs = np.array(xs), np.array(rs)
    mid = (xs > 4) & (xs < 28)
    slope, icpt = np.linalg.lstsq(np.stack([xs[mid], np.ones(mid.sum())], 1), rs[mid],
                                  rcond=None)[0]
    assert slope < 0
    dev = (rs - (slope * xs + icpt)) / abs(slope)       # in coarse cells of pressure drop
    assert np.abs(dev[mid]).max() < 0.25
    for last_coarse, first_fine in ((11.5, 12.25), (20.5, 19.75)):
        a = dev[np.isclose(xs, last_coarse)].mean()
        b = dev[np.isclose(xs, first_fine)].mean()
        assert abs(a - b) < 0.1, (interp, last_coarse, a, b)


# ---------------------------------------------------- momentum exchange
def _fluid_momentum(lbm, blocks):
    return sum((lbm.f[b][~lbm.solid[b]] @ lbm.vs.cf).sum(0) for b in blocks)


MEA_CASES = [
    ("2d_q9", lambda: W.periodic_box(dim=2, q=9, n=16, ny=16), 0),
    ("3d_q27", lambda: W.periodic_box(dim=3, q=27, n=16, ny=16, nz=8), 0),
    ("3d_q19_level1", lambda: W.periodic_box(dim=3, q=19, n=16, ny=16, nz=4,
                                             max_levels=2, max_blocks=64 * 9), 1),
]


@pytest.mark.parametrize("name,mk,level", MEA_CASES, ids=[c[0] for c in MEA_CASES])
def test_momentum_exchange_balances_fluid_momentum(name, mk, level):
    """Halfway bounce-back returns every post-collision population that meets
    the solid with the opposite velocity, while collision and streaming between
    fluid cells conserve momentum.  Over one update of a fully periodic level
    the fluid therefore loses exactly the momentum 2 sum f*_p c_p that the
    momentum exchange of Section 5.3 assigns to the solid: in lattice units of
    that level F / dx_L^(dim-1) = P(t) - P(t+1).  Pins the factor 2, the sign,
    the use of post-collision values, the link directions and dx_L."""
    cfg = mk()
    cfg["solid"] = (6.0, 10.0, 5.0, 11.0)
    lbm = ForestLBM(cfg)
    if level:
        m = np.zeros(lbm.mesh.cap, np.int8)
        m[:lbm.mesh.n_root] = 1
        lbm.adapt(m)
        assert lbm.mesh.counts()[level] == lbm.mesh.n_root * lbm.mesh.nc
    blocks = lbm.mesh.active_list(level)
    assert all(lbm.mesh.level[b] == level for b in blocks)
    for i, b in enumerate(blocks):
        rho, u = W.random_macro(100 + i, lbm.m, lbm.dim)
        f = equilibrium(lbm.vs, rho, u) + W.random_noise(5000 + i, (lbm.m, lbm.vs.q))
        f[lbm.solid[b]] = lbm.rest
        lbm.f[b] = f
    assert lbm.solid[blocks].any() and not lbm.solid[blocks].all()
    force = lbm.mea_force()
    p0 = _fluid_momentum(lbm, blocks)
    lbm.collide_stream(level)
    p1 = _fluid_momentum(lbm, blocks)
    dx = cfg["length_x"] / (cfg["nx"] * 2.0 ** level)
    lattice = force / dx ** (lbm.dim - 1)
    assert np.abs(lattice).max() > 1e-2
    np.testing.assert_allclose(lattice, p0 - p1, rtol=1e-10, atol=1e-11)


# ------------------------------------ exhaustive mark patterns, tiny forests
def _expected_decisions(mesh, geo, marks):
    """Refine and coarsen sets of one adaptation call, decided from geometry
    alone: a leaf below L_max - 1 marked +1 refines when every one of its
    same-level neighbour positions holds a block (walls count as present); a
    block marked -1 whose children are all leaves coarsens unless one of its
    children has, in some direction including itself, a same-level block that
    has children or refines in this call."""
    act = mesh.active_ids()
    refine = sorted(b for b in act if marks[b] > 0 and mesh.child0[b] == NONE
                    and mesh.level[b] < mesh.lmax - 1 and NONE not in geo[b])
    rset = set(refine)
    coarsen = []
    for p in sorted(act):
        c0 = mesh.child0[p]
        if marks[p] >= 0 or c0 < 0 or mesh.status[p] == REFINED_PERMANENT:
            continue
        kids = [c0 + c for c in range(mesh.nc)]
        if any(mesh.child0[c] >= 0 for c in kids):
            continue
        busy = any(n != "wall" and n != NONE and (mesh.child0[n] >= 0 or n in rset)
                   for c in kids for n in geo[c])
        if not busy:
            coarsen.append(p)
    return refine, coarsen


def _mesh_key(mesh):
    return tuple(sorted((int(mesh.level[b]), tuple(mesh.X[b]), int(mesh.status[b]))
                        for b in mesh.active_ids()))


def _check_call(mesh, marks, seen, classes):
    geo = {b: geometric_nbr(mesh, b) for b in mesh.active_ids()}
    refine, coarsen = _expected_decisions(mesh, geo, marks)
    gap_before = list(mesh.gap)
    child0_before = mesh.child0.copy()
    res = mesh.adapt(marks)
    assert not res["capacity_error"]
    assert (res["n_refined"], res["n_coarsened"]) == (len(refine), len(coarsen))
    for i, p in enumerate(refine):
        assert mesh.status[p] in REFINED_ANY
        assert mesh.child0[p] == gap_before[-1 - i * mesh.nc]
    for p in coarsen:
        assert mesh.status[p] == UNREFINED and mesh.child0[p] == NONE
    for b in np.flatnonzero(marks):
        if b not in refine and b not in coarsen:
            assert mesh.child0[b] == child0_before[b]
    brute_force_check(mesh)
    key = _mesh_key(mesh)
    if key in seen:
        return
    seen.add(key)
    for b in mesh.active_ids():
        g = geometric_nbr(mesh, b)
        for k, n in enumerate(g):
            assert mesh.nbr[b, k] <= -2 if n == "wall" else mesh.nbr[b, k] == n
        # a cell's class looks at most one block width away, so the block's
        # neighbour occupancy decides it: rasterise once per occupancy
        occ = tuple("wall" if n == "wall" else n != NONE for n in g)
        if occ not in classes:
            classes[occ] = brute_force_classes(mesh, b)
        assert np.array_equal(mesh.cell_classes(b), classes[occ])


def _effective_patterns(mesh):
    """Every mark pattern that can change the mesh: leaves 0 / +1, blocks with
    children 0 / -1."""
    act = sorted(mesh.active_ids())
    opts = [(0, 1) if mesh.child0[b] == NONE else (0, -1) for b in act]
    for combo in itertools.product(*opts):
        m = np.zeros(mesh.cap, np.int8)
        m[act] = combo
        yield m


EXHAUSTIVE = [
    ("2d_2x2", lambda: W.cavity(dim=2, n=8, max_levels=3, max_blocks=4 + 4 * 12),
     [(), (0,), (1,), (2,), (3,)]),
    ("3d_2x1x1", lambda: W.cavity(dim=3, n=8, ny=4, nz=4, max_levels=3,
                                  max_blocks=2 + 8 * 12), [(), (0,)]),
]


@pytest.mark.parametrize("name,mk,starts", EXHAUSTIVE, ids=[e[0] for e in EXHAUSTIVE])
def test_exhaustive_mark_patterns(name, mk, starts):
    """Every mark pattern (-1 / 0 / +1) on the roots, then every pattern that
    can change the mesh on the forests with the listed roots refined: the
    refine / coarsen decisions equal the geometric rule, the group heads follow
    the gap stack, and the invariants hold after every call."""
    cfg = mk()
    n_root = Forest(cfg).n_root
    seen, classes = set(), {}
    for pat in itertools.product((-1, 0, 1), repeat=n_root):
        mesh = Forest(cfg)
        m = np.zeros(mesh.cap, np.int8)
        m[:n_root] = pat
        _check_call(mesh, m, seen, classes)
        refined = tuple(b for b in range(n_root) if mesh.child0[b] >= 0)
        assert refined == tuple(b for b in range(n_root) if pat[b] == 1)
    n_calls = 0
    for refined in starts:
        start = Forest(cfg)
        m = np.zeros(start.cap, np.int8)
        m[list(refined)] = 1
        start.adapt(m)
        for m2 in _effective_patterns(start):
            _check_call(copy.deepcopy(start), m2, seen, classes)
            n_calls += 1
    nc = Forest(cfg).nc
    assert n_calls == sum(2 ** (n_root + len(r) * nc) for r in starts)
    assert len(seen) > 10

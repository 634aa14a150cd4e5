"""Full-size GPU parity, in the launch configuration the benchmark times (CUDA
graphs, default collide-stream kernel):

* the complete 2D cavity run: 64 x 64 root cells, D2Q9, FP64, L_max 3, Re 100,
  2000 coarse steps with the vorticity criterion every 100 steps;
* one coarse step of the 3D cavity at 64^3 root cells, D3Q19, FP32, L_max 4,
  capacity 524,288 blocks, on a four-level layered mesh (213,696 blocks) from
  a seeded state;
* the same cavity cut to 32^3 root cells (Re 1000, L_max 4): 150 coarse steps
  from rest with the criterion every 50, in FP64 (adapting on its own
  criterion) and in FP32 (adapting with the oracle's marks, since an FP32
  criterion may fall on the other side of a threshold).

The expected values are written by `golden/make_fullsize.py`, which runs the
oracle alone: SHA-256 digests of the mesh tables (bit-exact: block, neighbour,
ID-set and gap tables, coordinates, cell classes) after every adaptation, and
the populations of sampled blocks of every level (leaves at a coarse-fine
boundary, interior leaves, refined blocks that receive averaged values):
relative L2 <= 1e-12 in FP64 and <= 1e-5 in FP32 per level, over the cells
that carry the method's result (the cells of refined blocks over interior
children are covered: neither read nor written by the method, they hold
left-over values that the push and the pull form of streaming leave
differently)."""
import os

import numpy as np
import pytest

import fullsize_cases as FC
import workloads as W
from cellwise import assert_cells
from oracle.lattice import VelocitySet, equilibrium, velocities

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def per_level_errors(gpu, ids, want, lmax, storage):
    """Relative L2 per level over the cells of the sampled blocks that carry
    the method's result (covered cells of refined blocks are left over), and
    the same split into leaves and refined blocks for the message.  The worst
    cell of each class (ghost, interface, interior) is held to the per-cell
    bar as well."""
    blk = gpu.blocks()
    masks = gpu.masks()
    valid = FC.valid_cells(ids, blk["status"], blk["child0"], masks, gpu.dim)
    got = gpu.populations()[ids]
    vs = VelocitySet(gpu.dim, gpu.q)
    assert_cells(got, want, masks[ids], vs.w, storage, valid=valid, what="sampled blocks")
    levels = blk["level"][ids]
    leaf = blk["status"][ids] == 1
    with_leaves = set(blk["level"][blk["status"] == 1].tolist())
    assert with_leaves <= set(levels.tolist())       # every level that holds leaves is sampled
    populated = sorted(set(levels.tolist()))

    def rel(sel):
        if not np.any(sel):
            return None
        return float(np.linalg.norm(got[sel] - want[sel]) / np.linalg.norm(want[sel]))

    out, detail = {}, {}
    for L in populated:
        lev = (levels == L)[:, None] & valid
        out[L] = rel(lev)
        detail[L] = (rel(lev & leaf[:, None]), rel(lev & ~leaf[:, None]))
    return out, detail


def test_cavity2d_full_run_matches_oracle(golden_dir):
    from paper_2308_08085_gb300 import AmrLBM
    want = np.load(os.path.join(golden_dir, "c0_full_run.npz"))
    cfg = FC.c0_config()
    gpu = AmrLBM(cfg, storage="f64")
    for t in range(FC.C0_PERIODS):
        gpu.step(FC.C0_EVERY)
        gpu.adapt()
        assert gpu.counts()["n_ids"] == want["counts"][t].tolist(), t
        assert FC.gpu_digest(gpu) == str(want["digests"][t]), "mesh tables differ after adaptation %d" % t
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"], "f64")
    assert max(err.values()) <= 1e-12, detail
    gpu.close()


def test_cavity3d_full_size_step_matches_oracle(golden_dir):
    from paper_2308_08085_gb300 import AmrLBM
    want = np.load(os.path.join(golden_dir, "c1_full_step.npz"))
    cfg = FC.c1_config()
    gpu = AmrLBM(cfg, storage="f32", kernel_variant=0)
    for r in range(len(FC.C1_SLABS)):
        blk = gpu.blocks()
        m = FC.c1_marks(blk["level"], blk["status"], gpu.coords()[:, 2], r)
        rc, _ = gpu.adapt(torch.from_numpy(m).cuda())
        assert rc == 0
    assert gpu.counts()["n_ids"] == want["counts"].tolist()
    assert FC.gpu_digest(gpu) == str(want["digest"]), "mesh tables differ"
    vs = VelocitySet(3, 19)
    rest = equilibrium(vs, np.ones(1), np.zeros((1, 3)))[0]
    f = FC.seeded_state(vs, rest, gpu.id_sets(), gpu.cap, gpu.m, FC.C1_STATE_SEED)
    gpu.set_populations(f)
    del f
    gpu.step(1)
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"], "f32")
    assert max(err.values()) <= 1e-5, detail
    gpu.close()


def test_cavity3d_cut_run_matches_oracle(golden_dir):
    from paper_2308_08085_gb300 import AmrLBM
    want = np.load(os.path.join(golden_dir, "c1cut_run.npz"))
    cfg = FC.c1cut_config()
    gpu = AmrLBM(cfg, storage="f64")
    for t in range(FC.C1CUT_PERIODS):
        gpu.step(FC.C1CUT_EVERY)
        gpu.adapt()
        assert gpu.counts()["n_ids"] == want["counts"][t].tolist(), t
        assert FC.gpu_digest(gpu) == str(want["digests"][t]), "mesh tables differ after adaptation %d" % t
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"], "f64")
    assert max(err.values()) <= 1e-12, detail
    gpu.close()
    gpu = AmrLBM(cfg, storage="f32")
    for t in range(FC.C1CUT_PERIODS):
        gpu.step(FC.C1CUT_EVERY)
        gpu.adapt(torch.from_numpy(np.ascontiguousarray(want["marks"][t])).cuda())
        assert FC.gpu_digest(gpu) == str(want["digests"][t]), t
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"], "f32")
    assert max(err.values()) <= 1e-5, detail
    gpu.close()


def forest_invariants(gpu, dim):
    """Properties every forest satisfies at any size, checked on the exported
    tables: the leaves tile the domain; every same-level neighbour link lands
    on the block at the geometric offset (periodic wrap) and is mirrored by
    the opposite link; a missing neighbour of a child (NONE) means that the
    parent has a neighbour there (2:1 balance)."""
    blk = gpu.blocks()
    lev, st, par = blk["level"], blk["status"], blk["parent"]
    X, nbr = gpu.coords(), gpu.nbr().astype(np.int64)
    cfg = gpu.cfg
    ext = np.array([cfg["nx"], cfg["ny"], cfg["nz"]][:dim], np.float64)
    alive = np.nonzero(st > 0)[0]
    leaves = alive[st[alive] == 1]
    assert np.isclose(((4.0 / 2.0 ** lev[leaves]) ** dim).sum(), np.prod(ext))
    c = velocities(dim, 9 if dim == 2 else 27)
    opp = np.array([int(np.nonzero((c == -c[k]).all(1))[0][0]) for k in range(len(c))])
    k_of_code = np.zeros(27, np.int64)
    for k in range(len(c)):
        k_of_code[(c[k, 0] + 1) + 3 * (c[k, 1] + 1) + (9 * (c[k, 2] + 1) if dim == 3 else 0)] = k
    periodic = np.array([cfg["faces"][2 * a][0] == "periodic" for a in range(dim)])
    for k in range(1, len(c)):
        nb = nbr[alive, k]
        ok = nb >= 0
        src, dst = alive[ok], nb[ok]
        assert np.all(lev[dst] == lev[src]), k
        want = X[src] + c[k] * (4.0 / 2.0 ** lev[src])[:, None]
        want = np.where(periodic, np.mod(want, ext), want)
        assert np.array_equal(X[dst], want), k
        assert np.all(nbr[dst, opp[k]] == src), k
        # 2:1: where a child has no same-level neighbour, the parent level has
        # a block (or a wall) at that position
        none = alive[(nb == -1) & (lev[alive] > 0)]
        if len(none):
            wc = (4.0 / 2.0 ** lev[none])[:, None]
            P = par[none]
            off = np.floor((X[none] + c[k] * wc - X[P]) / (2.0 * wc)).astype(np.int64)
            code = (off[:, 0] + 1) + 3 * (off[:, 1] + 1) + (9 * (off[:, 2] + 1) if dim == 3 else 0)
            assert np.all(nbr[P, k_of_code[code]] != -1), k


def test_cylinder_full_size_mesh_invariants_and_rest_prism():
    """The prism configuration at full size (256 x 64 x 64 root cells, D3Q27,
    L_max 5, capacity 4,000,000 blocks), built as the benchmark builds it
    (five adaptations of the frozen distance rule): forest invariants over
    the 3.5 million blocks; then one coarse step in FP16 storage (default
    launch configuration) leaves every solid cell at the rest state."""
    from paper_2308_08085_gb300 import AMR_RHO_U, AmrLBM
    cfg = W.channel_cylinder(q=27, nx=256, ny=64, nz=64, side=8, cx=64, cy=32, max_levels=5,
                             crit_start=100, crit_inc=1, max_blocks=4_000_000)
    gpu = AmrLBM(cfg, storage="f16")
    for _ in range(5):
        rc, _ = gpu.adapt()
        assert rc == 0
    counts = gpu.counts()["n_ids"]
    assert counts == [16384, 63488, 211968, 694272, 2568192]
    forest_invariants(gpu, 3)
    gpu.step(1)
    ru = gpu.fields_device(AMR_RHO_U, torch.float64).reshape(gpu.cap, gpu.m, 4)
    blk = gpu.blocks()
    X = gpu.coords()
    x0, x1, y0, y1 = cfg["solid"]
    lc = np.array([[l % 4, (l // 4) % 4, l // 16] for l in range(64)], np.float64)
    leaves = np.nonzero(blk["status"] == 1)[0]
    near = leaves[(X[leaves, 0] < x1 + 1) & (X[leaves, 0] + 4 > x0 - 1)
                  & (X[leaves, 1] < y1 + 1) & (X[leaves, 1] + 4 > y0 - 1)]
    sub = ru[torch.from_numpy(near).to(ru.device)].cpu().numpy()     # [n, 64, 4]
    solid_cells = 0
    for r, b in enumerate(near):
        h = 1.0 / 2.0 ** blk["level"][b]
        ctr = X[b] + (lc + 0.5) * h
        sol = (ctr[:, 0] > x0) & (ctr[:, 0] < x1) & (ctr[:, 1] > y0) & (ctr[:, 1] < y1)
        solid_cells += int(sol.sum())
        # the rest equilibrium, up to the rounding of the FP32 moments
        assert np.all(np.abs(sub[r, sol, 0] - 1.0) <= 1e-6), b
        assert np.all(np.abs(sub[r, sol, 1:]) <= 1e-7), b
    assert solid_cells > 1000
    del ru
    gpu.close()


def test_batched_cavities_full_size_equal_individual_runs():
    """The 64 batched cavities of the benchmark at full size (their root grids,
    depths and capacities): after refining two block layers under the lid on
    every level, one period of 50 coarse steps advanced by the batch in the
    graph form, then one more in one persistent launch, equals the same
    instances advanced one by one, to rounding (the batched and the
    per-instance kernels are compiled separately); a third period in the
    member-graph form, started from the individually advanced state, runs
    the per-instance kernels as branches of one graph and equals them to the
    bit."""
    from paper_2308_08085_gb300 import AMR_F, AmrBatch, AmrLBM
    cfgs = W.batched_cavities(64, seed=0)

    def build():
        sims = [AmrLBM(c, storage="f32") for c in cfgs]
        for i, sim in enumerate(sims):
            for r in range(sim.lmax - 1):      # two block layers under the lid per level
                blk = sim.blocks()
                h = 4.0 / 2 ** r
                m = W.slab_marks(blk["level"], blk["status"], sim.coords()[:, 2], r, h,
                                 cfgs[i]["nz"] - h, h, 0.0, 1000 + 10 * i + r)
                rc, _ = sim.adapt(torch.from_numpy(m).cuda())
                assert rc == 0
        return sims

    batched, single = build(), build()
    batch = AmrBatch(batched)

    def compare():
        # a member that is BGK-unstable (tau_0 near 1/2 on a 32^3 root grid
        # at Re near 3200) diverges, and there any rounding difference grows
        # without bound: members whose populations leave [-2, 2] on either
        # side are counted, not compared
        worst, diverged = 0.0, 0
        for a, b in zip(batched, single):
            assert a.counts()["n_ids"] == b.counts()["n_ids"]
            fa = a.fields_device(AMR_F, torch.float64)
            fb = b.fields_device(AMR_F, torch.float64)
            bounded = bool(torch.isfinite(fa).all() and torch.isfinite(fb).all() and
                           fa.abs().max() < 2 and fb.abs().max() < 2)
            if bounded:
                worst = max(worst, float(torch.linalg.norm(fa - fb) / torch.linalg.norm(fb)))
            else:
                diverged += 1
            del fa, fb
        assert diverged <= 16, diverged
        return worst

    batch.step(50)                             # graph form
    for sim in single:
        sim.step(50)
    worst = compare()
    assert worst <= 1e-6, worst
    batch.configure("persistent", 128, 2)      # then 50 steps in one persistent launch
    batch.step(50)
    batch.sync()
    for sim in single:
        sim.step(50)
    worst = compare()
    assert worst <= 1e-6, worst
    # then 50 in the member-graph form, from the individually advanced state:
    # the members' own kernels as branches of one graph, so equal to the bit
    for a, b in zip(batched, single):
        a.restore(b.checkpoint())
    batch.configure("members")
    batch.step(50)
    for sim in single:
        sim.step(50)
    for a, b in zip(batched, single):       # bit patterns (a diverged member may hold NaN)
        assert torch.equal(a.fields_device(AMR_F, torch.float64).view(torch.int64),
                           b.fields_device(AMR_F, torch.float64).view(torch.int64))
    assert sum(sum(s.counts()["n_ids"]) for s in single) > 500_000
    batch.close()
    for sim in batched + single:
        sim.close()

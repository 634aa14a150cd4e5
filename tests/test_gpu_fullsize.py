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
from oracle.lattice import VelocitySet, equilibrium

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def per_level_errors(gpu, ids, want, lmax):
    """Relative L2 per level over the cells of the sampled blocks that carry
    the method's result (covered cells of refined blocks are left over), and
    the same split into leaves and refined blocks for the message."""
    blk = gpu.blocks()
    valid = FC.valid_cells(ids, blk["status"], blk["child0"], gpu.masks(), gpu.dim)
    got = gpu.populations()[ids]
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
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"])
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
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"])
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
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"])
    assert max(err.values()) <= 1e-12, detail
    gpu.close()
    gpu = AmrLBM(cfg, storage="f32")
    for t in range(FC.C1CUT_PERIODS):
        gpu.step(FC.C1CUT_EVERY)
        gpu.adapt(torch.from_numpy(np.ascontiguousarray(want["marks"][t])).cuda())
        assert FC.gpu_digest(gpu) == str(want["digests"][t]), t
    err, detail = per_level_errors(gpu, want["ids"], want["f"], cfg["max_levels"])
    assert max(err.values()) <= 1e-5, detail
    gpu.close()

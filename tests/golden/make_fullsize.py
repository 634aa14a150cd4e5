"""Writes the expected values of the full-size parity cases (the cases are
defined in tests/fullsize_cases.py) by running the oracle alone.

    python tests/golden/make_fullsize.py [c0] [c1] [c1cut]

c0_full_run.npz: the mesh-table digest and per-level block counts after each
  of the 20 adaptations of the 2D cavity run, the sampled block IDs, and their
  populations at the end of the run (after the last adaptation).
c1_full_step.npz: the digest and counts of the layered 3D mesh, the sampled
  block IDs and their populations after one coarse step from the seeded state.
c1cut_run.npz: the 3D cavity cut to 32^3 root cells, 150 coarse steps from
  rest with the criterion every 50: the criterion's marks, digests and counts
  of each adaptation, sampled blocks at the end.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]

import numpy as np  # noqa: E402

import fullsize_cases as FC  # noqa: E402
from oracle.solver import ForestLBM  # noqa: E402


def c0():
    cfg = FC.c0_config()
    ref = ForestLBM(cfg)
    digests, counts = [], []
    for t in range(FC.C0_PERIODS):
        ref.step(FC.C0_EVERY)
        ref.adapt()
        digests.append(FC.oracle_digest(ref.mesh))
        counts.append(ref.mesh.counts())
        print("c0 period %d counts %s" % (t, counts[-1]), flush=True)
    mesh = ref.mesh
    ids = FC.sample_blocks(mesh.level, mesh.status, mesh.child0, mesh.nbr, mesh.lmax, mesh.nc,
                           FC.C0_SAMPLE_SEED)
    np.savez_compressed(os.path.join(HERE, "c0_full_run.npz"), digests=np.array(digests),
                        counts=np.array(counts, np.int64), ids=ids, f=ref.f[ids])


def c1cut():
    cfg = FC.c1cut_config()
    ref = ForestLBM(cfg)
    digests, counts, marks = [], [], []
    for t in range(FC.C1CUT_PERIODS):
        ref.step(FC.C1CUT_EVERY)
        ref.sync()
        m, _ = ref.criterion_marks()
        marks.append(np.asarray(m, np.int8))
        ref.adapt(m)
        digests.append(FC.oracle_digest(ref.mesh))
        counts.append(ref.mesh.counts())
        print("c1cut period %d counts %s" % (t, counts[-1]), flush=True)
    mesh = ref.mesh
    ids = FC.sample_blocks(mesh.level, mesh.status, mesh.child0, mesh.nbr, mesh.lmax, mesh.nc,
                           FC.C1CUT_SAMPLE_SEED)
    np.savez_compressed(os.path.join(HERE, "c1cut_run.npz"), digests=np.array(digests),
                        counts=np.array(counts, np.int64), marks=np.array(marks), ids=ids,
                        f=ref.f[ids])


def c1():
    cfg = FC.c1_config()
    ref = ForestLBM(cfg)
    mesh = ref.mesh
    for r in range(len(FC.C1_SLABS)):
        res = mesh.adapt(FC.c1_marks(mesh.level, mesh.status, mesh.X[:, 2], r))
        assert not res["capacity_error"]
        print("c1 round %d counts %s" % (r, mesh.counts()), flush=True)
    digest = FC.oracle_digest(mesh)
    ref.f = FC.seeded_state(ref.vs, ref.rest, mesh.id_sets, mesh.cap, ref.m, FC.C1_STATE_SEED)
    ids = FC.sample_blocks(mesh.level, mesh.status, mesh.child0, mesh.nbr, mesh.lmax, mesh.nc,
                           FC.C1_SAMPLE_SEED)
    t = time.time()
    ref.step(1)
    print("c1 step %.1f s" % (time.time() - t), flush=True)
    np.savez_compressed(os.path.join(HERE, "c1_full_step.npz"), digest=np.array(digest),
                        counts=np.array(mesh.counts(), np.int64), ids=ids, f=ref.f[ids])


if __name__ == "__main__":
    which = sys.argv[1:] or ["c0", "c1", "c1cut"]
    for w in which:
        {"c0": c0, "c1": c1, "c1cut": c1cut}[w]()

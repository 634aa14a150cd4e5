"""Batched instances: several forests of different sizes and depths advanced
together -- in the graph form (one launch per level operation), in the
persistent form (one launch whose work queue walks the level order with
per-member dependency counters) for several tile shapes, and in the
member-graph form (the members' own coarse steps as branches of one graph)
-- must give the
populations of the same forests advanced one by one: the same arithmetic per
cell, compiled into different kernels, so equal up to the compiler's fused
multiply-add choices (rounding-level differences).  One member of each form
must match the CPU oracle, and the persistent form's bounded waits must give
up and report it when no wait can be satisfied."""
import numpy as np
import pytest

import workloads as W
from cellwise import assert_cells, oracle_classes
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


CFGS = [
    lambda: W.cavity(dim=3, q=19, n=8, max_levels=2, re=200.0, max_blocks=8 * 12),
    lambda: W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=3, re=400.0, max_blocks=12 * 40),
    lambda: W.cavity(dim=3, q=19, n=16, max_levels=1, re=800.0, max_blocks=64),
]


def member(cfg, storage, marks_seq, state):
    from paper_2308_08085_gb300 import AmrLBM
    m = AmrLBM(cfg, storage=storage)
    for mk in marks_seq:
        m.adapt(torch.from_numpy(mk).cuda())
    m.set_populations(state)
    return m


def seeded(cfg, seed):
    """Marks (two rounds) and a random state for a config, from the oracle
    mesh so that the same marks apply to every copy."""
    ref = ForestLBM(cfg)
    seq = []
    for r in range(2):
        mk = np.zeros(cfg["max_blocks"], np.int8)
        leaves = [b for b in ref.mesh.active_ids() if ref.mesh.status[b] == 1]
        mk[leaves[: max(1, len(leaves) // 3)]] = 1
        ref.adapt(mk)
        seq.append(mk)
    n = cfg["max_blocks"] * ref.m
    rho, u = W.random_macro(seed, n, 3)
    f = equilibrium(ref.vs, rho, u) + W.random_noise(seed + 1, (n, ref.vs.q), 1e-3)
    f = f.reshape(cfg["max_blocks"], ref.m, ref.vs.q)
    ref.f[:] = f
    return ref, seq, f


ROUNDING = {"f32": 1e-6, "f64": 1e-13}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


FORMS = [("graph", 512, 0), ("graph", 64, 0), ("persistent", 64, 1), ("persistent", 128, 2),
         ("persistent", 256, 8), ("members", 0, 0)]


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("form", FORMS, ids=["%s-%d-%d" % f for f in FORMS])
def test_batch_equals_individual_runs(storage, form):
    from paper_2308_08085_gb300 import AmrBatch
    cfgs = [mk() for mk in CFGS]
    data = [seeded(c, 40 + i) for i, c in enumerate(cfgs)]
    batched = [member(c, storage, seq, f) for c, (_, seq, f) in zip(cfgs, data)]
    single = [member(c, storage, seq, f) for c, (_, seq, f) in zip(cfgs, data)]
    batch = AmrBatch(batched)
    batch.configure(*form)
    l0 = batch.launches()
    batch.step(3)
    if form[0] == "persistent":
        assert batch.launches() - l0 == 1          # three coarse steps, one launch
    batch.sync()
    for m in single:
        m.step(3)
    for b, s in zip(batched, single):
        assert rel(b.populations(), s.populations()) <= ROUNDING[storage]
    # adapt every member with its criterion, re-batch and continue
    for b, s in zip(batched, single):
        b.adapt()
        s.adapt()
    batch.refresh()
    batch.step(2)
    batch.sync()
    for m in single:
        m.step(2)
    for b, s in zip(batched, single):
        assert rel(b.populations(), s.populations()) <= ROUNDING[storage]
        assert np.array_equal(b.blocks()["status"], s.blocks()["status"])
    # a member stepped outside the batch breaks lock-step: refused
    batched[0].step(1)
    from paper_2308_08085_gb300.amr import AmrError
    with pytest.raises(AmrError):
        batch.step(1)
    batch.close()


def test_batch_member_matches_oracle_and_autotune():
    from paper_2308_08085_gb300 import AmrBatch
    from paper_2308_08085_gb300.amr import BATCH_CANDIDATES
    cfgs = [mk() for mk in CFGS]
    data = [seeded(c, 60 + i) for i, c in enumerate(cfgs)]
    members = [member(c, "f64", seq, f) for c, (_, seq, f) in zip(cfgs, data)]
    batch = AmrBatch(members)
    # 17 candidates x (1 + 1) coarse steps, then one more
    chosen, times = batch.autotune(trial_steps=1)
    assert sorted(times) == sorted(BATCH_CANDIDATES) and all(v > 0 for v in times.values())
    assert chosen["form"] in ("graph", "persistent", "members")
    assert (chosen["form"], chosen["threads"], chosen["tile_blocks"]) in times
    assert times[(chosen["form"], chosen["threads"], chosen["tile_blocks"])] == min(times.values())
    batch.step(1)
    batch.sync()
    ref = data[1][0]
    ref.step(35)
    ref.sync()
    members[1].rho_u()
    ids = ref.mesh.active_ids()
    got = members[1].populations()[ids]
    err = np.linalg.norm(got - ref.f[ids]) / np.linalg.norm(ref.f[ids])
    assert err <= 1e-12, err
    assert_cells(got, ref.f[ids], oracle_classes(ref.mesh, ids), ref.vs.w, "f64")
    assert batch.launches() > 0
    batch.close()


@pytest.mark.parametrize("tile", [(64, 1), (256, 4)])
def test_persistent_member_matches_oracle(tile):
    """FP64, persistent form: members 1 and 2 after five coarse steps (one
    launch) against the oracle at 1e-12, per cell at 1e-10, after the level
    synchronisation on both sides.  (Member 0 has every root refined and no
    interface: its roots hold no solution, and their stored values are not
    the oracle's.)"""
    from paper_2308_08085_gb300 import AmrBatch
    cfgs = [mk() for mk in CFGS]
    data = [seeded(c, 80 + i) for i, c in enumerate(cfgs)]
    members = [member(c, "f64", seq, f) for c, (_, seq, f) in zip(cfgs, data)]
    batch = AmrBatch(members)
    batch.configure("persistent", tile[0], tile[1])
    batch.step(5)
    batch.sync()
    for i in (1, 2):
        ref = data[i][0]
        ref.step(5)
        ref.sync()
        members[i].rho_u()                     # the level synchronisation, as ref.sync()
        ids = ref.mesh.active_ids()
        got = members[i].populations()[ids]
        err = np.linalg.norm(got - ref.f[ids]) / np.linalg.norm(ref.f[ids])
        assert err <= 1e-12, (i, err)
        assert_cells(got, ref.f[ids], oracle_classes(ref.mesh, ids), ref.vs.w, "f64")
    batch.close()


def test_persistent_bounded_wait_reports_timeout():
    """No wait of the launch can be satisfied: every wait gives up after its
    limit, the launch ends, amr_batch_sync reports AMR_E_TIMEOUT once, and
    the members' own synchronising calls are clear afterwards."""
    from paper_2308_08085_gb300 import AmrBatch
    from paper_2308_08085_gb300.amr import AMR_E_TIMEOUT, AMR_E_INVAL
    cfgs = [mk() for mk in CFGS]
    data = [seeded(c, 90 + i) for i, c in enumerate(cfgs)]
    members = [member(c, "f32", seq, f) for c, (_, seq, f) in zip(cfgs, data)]
    batch = AmrBatch(members)
    assert batch.check_timeout(1 << 20) == AMR_E_INVAL     # graph form: refused
    batch.configure("persistent", 128, 2)
    assert batch.check_timeout(1 << 20) == AMR_E_TIMEOUT
    batch.sync()                                           # reported once
    for m in members:
        m.mass()                                           # no pending wait flag
    batch.close()


def test_batch_rejects_cubic_members():
    from paper_2308_08085_gb300 import AmrBatch, AmrLBM
    from paper_2308_08085_gb300.amr import AmrError
    cfg = W.cavity(dim=3, q=19, n=8, max_levels=2, max_blocks=8 * 12)
    cfg["interp"] = "cubic"
    m = AmrLBM(cfg, storage="f32")
    with pytest.raises(AmrError):
        AmrBatch([m])
    m.close()

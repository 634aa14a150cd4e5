"""Device validation of the block tables (amr_check_tables, amr_validate_tables),
the stand-in for a device bounds checker.

* Valid inputs: instances created with check_tables = 1 (the validation runs
  at amr_init and after every amr_adapt, and fails the call on a bad entry)
  go through refinement, coarsening, the criterion and the distance rule in
  2D and 3D, with and without a solid prism; every call succeeds and a final
  amr_check_tables finds no bad entry.
* Detection: amr_validate_tables on copies of an instance's exported tables
  finds nothing, and finds one bad entry, at the right block and with the
  right check, in each copy where one entry was changed.  The changed tables
  are only read by the validator, which dereferences an index only after
  finding it in range; no simulation kernel ever sees them.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NONE = -1
CHECK = dict(STATUS=1, INACTIVE=2, LEVEL=3, SELF=4, NEIGHBOUR=5, UNUSED=6, CHILDREN=7,
             PARENT=8, GAP=9, LIST=10, GROUP=11)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def checked(cfg, storage="f64"):
    from paper_2308_08085_gb300 import AmrLBM
    cfg = dict(cfg)
    cfg["check_tables"] = 1
    return AmrLBM(cfg, storage=storage)


def cycle(sim, seed, rounds=3):
    """Random refine / coarsen marks, then the criterion, each followed by a
    few steps; every adaptation validates the tables."""
    for r in range(rounds):
        marks = W.random_marks(seed + r, sim.cap)
        rc, _ = sim.adapt(torch.from_numpy(marks).cuda())
        assert rc in (0, -2)                          # AMR_OK or AMR_E_CAPACITY
        sim.step(2)
    sim.adapt()
    sim.step(2)


CASES = {
    "cavity2d": lambda: W.cavity(dim=2, q=9, n=24, max_levels=3, max_blocks=36 + 4 * 60),
    "cavity3d": lambda: W.cavity(dim=3, q=19, n=16, max_levels=3, max_blocks=64 + 8 * 60),
    "cylinder3d": lambda: W.channel_cylinder(q=19, nx=64, ny=16, nz=16, side=4, cx=16, cy=8,
                                              max_levels=3, max_blocks=256 + 8 * 200),
    "cylinder2d": lambda: W.channel_cylinder(dim=2, nx=96, ny=48, side=8, cx=24, cy=24,
                                              refine_dist=0.05, max_levels=3,
                                              max_blocks=288 + 4 * 300),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_checked_instances_stay_valid(name):
    sim = checked(CASES[name]())
    cycle(sim, seed=17)
    bad, first, code = sim.check_tables()
    assert (bad, first, code) == (0, -1, 0)
    sim.close()


def exported(sim):
    """Device copies of the tables in the validator's input layout."""
    from paper_2308_08085_gb300 import AMR_BLOCKS, AMR_GAPS, AMR_NBR
    blk = sim.fields_device(AMR_BLOCKS, torch.int32).reshape(4, sim.cap)
    nbr = sim.fields_device(AMR_NBR, torch.int32).reshape(sim.cap, sim.nk)
    row = torch.full((sim.cap, 32), NONE, dtype=torch.int32, device=nbr.device)
    row[:, :sim.nk] = nbr
    gaps = torch.tensor(sim.gaps(), dtype=torch.int32, device=nbr.device)
    return {"level": blk[0].clone(), "status": blk[1].clone(), "child0": blk[2].clone(),
            "parent": blk[3].clone(), "nbr": row, "gap": gaps}


def validate(sim, t):
    from paper_2308_08085_gb300.amr import validate_tables
    return validate_tables(sim.dim, sim.lmax, t["level"], t["status"], t["child0"],
                           t["parent"], t["nbr"], t["gap"] if t["gap"].numel() else None)


def test_validator_finds_each_planted_entry():
    sim = checked(CASES["cavity3d"]())
    marks = np.zeros(sim.cap, np.int8)
    marks[[5, 6, 9, 10, 21, 22, 25, 26]] = 1           # a 2x2x2 group of the 4x4x4 roots
    sim.adapt(torch.from_numpy(marks).cuda())
    tab = exported(sim)
    assert validate(sim, tab) == (0, -1, 0)
    lev = tab["level"].cpu().numpy()
    st = tab["status"].cpu().numpy()
    c0 = tab["child0"].cpu().numpy()
    leaf1 = int(np.nonzero((lev == 1) & (st == 1))[0][0])   # a level-1 leaf
    root = 0                                             # a level-0 leaf with neighbours
    refined = 5
    inactive = int(tab["gap"][0])

    def planted(field, index, value):
        t = {k: v.clone() for k, v in tab.items()}
        t[field][index] = value
        return t

    cases = [
        (planted("nbr", (root, 1), sim.cap + 5), root, "NEIGHBOUR"),   # out of range
        (planted("nbr", (leaf1, 4), 0), leaf1, "NEIGHBOUR"),           # another level
        (planted("nbr", (root, 0), 1), root, "SELF"),
        (planted("nbr", (root, 30), 3), root, "UNUSED"),
        (planted("child0", refined, sim.cap - 2), refined, "CHILDREN"),  # past the end
        (planted("child0", refined, int(c0[refined]) + 8), refined, "CHILDREN"),
        (planted("parent", leaf1, NONE), leaf1, "PARENT"),
        (planted("level", root, 7), root, "LEVEL"),
        (planted("status", root, 9), root, "STATUS"),
        (planted("level", inactive, 0), inactive, "INACTIVE"),
        (planted("gap", 0, root), root, "GAP"),                        # an active block
    ]
    for t, block, what in cases:
        bad, first, code = validate(sim, t)
        assert bad >= 1 and first <= block, (what, bad, first, code)
        if first == block:
            assert code == CHECK[what], (what, bad, first, code)
    # entries whose failure shows only at the block itself: exactly one
    for t, what in [(planted("status", root, 9), "STATUS"), (planted("nbr", (root, 0), 1), "SELF"),
                    (planted("nbr", (root, 1), sim.cap + 5), "NEIGHBOUR"),
                    (planted("gap", 0, root), "GAP")]:
        assert validate(sim, t) == (1, root, CHECK[what]), what
    sim.close()

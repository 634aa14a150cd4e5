"""Host logic of the persistent batched form (amr_batch_plan, no GPU): the
phase list, the tiles and the dependencies that the device work queue
follows, against an independent statement of the rules.

* Phases: the recursive level step (Section 4.1) of the batch, interpolation
  into level L+1 (when some member has level L+1 and exchanging parents on
  L), collide-stream of L (when some member has active blocks there), the
  two substeps of L+1, then averaging of L+1 into L; the buffer of a level
  is its parity bit at that moment, each collide-stream flipping it.
* Tiles: M_L blocks per collide-stream tile, threads / 4^D parents per
  interpolation tile, threads / 4^D children per averaging tile, member by
  member.
* Dependencies: each member waits for its own previous phase with tiles,
  cyclically (the previous coarse step when none comes before).  So every
  tile depends only on tiles earlier in the queue order (step, phase,
  member, tile): the earliest unfinished tile can always run.
"""
import ctypes

import numpy as np
import pytest

INTERP, COLLIDE, AVERAGE = 0, 1, 2


@pytest.fixture(scope="module")
def lib():
    from paper_2308_08085_gb300 import build as b
    from paper_2308_08085_gb300.amr import load_library
    return load_library(b.build())


def expected_phases(lmax, ids, act, par, cur):
    """(kind, level, buffer of the level, buffer of level + 1) in order."""
    out = []
    state = [cur]

    def rec(L):
        fine = L + 1 < lmax and ids[:, L + 1].sum() > 0
        np_ = par[:, L].sum()
        c = state[0]
        if fine and np_ > 0:
            out.append((INTERP, L, (c >> L) & 1, (c >> (L + 1)) & 1))
        if act[:, L].sum() > 0:
            out.append((COLLIDE, L, (c >> L) & 1, 0))
        state[0] ^= 1 << L
        if fine:
            rec(L + 1)
            rec(L + 1)
            if np_ > 0:
                c = state[0]
                out.append((AVERAGE, L, (c >> L) & 1, (c >> (L + 1)) & 1))

    rec(0)
    return out


def member_tiles(kind, L, i, member_lmax, act, par, dim, threads, tile):
    if L >= member_lmax[i]:
        return 0
    m, nc = (16, 4) if dim == 2 else (64, 8)
    u = threads // m
    if kind == COLLIDE:
        return -(-act[i, L] // tile)
    if kind == INTERP:
        return -(-par[i, L] // u)
    return -(-(par[i, L] * nc) // u)


def call_plan(lib, dim, member_lmax, ids, act, par, threads, tile, cur, max_phases=64):
    n, lmax = ids.shape
    ml = np.ascontiguousarray(member_lmax, np.int32)
    ids_, act_, par_ = (np.ascontiguousarray(a, np.int64) for a in (ids, act, par))
    n_phase = np.zeros(1, np.int32)
    phases = np.zeros(4 * max_phases, np.int32)
    toff = np.zeros(max_phases * (n + 1), np.int32)
    dep = np.zeros(max_phases * n, np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.amr_batch_plan(dim, n, lmax, ptr(ml), ptr(ids_), ptr(act_), ptr(par_), threads, tile,
                            cur, max_phases, ptr(n_phase), ptr(phases), ptr(toff), ptr(dep))
    return rc, int(n_phase[0]), phases, toff, dep


# three members: one level only; three levels with refinement on both; two levels
MEMBER_LMAX = [1, 3, 2]
IDS = np.array([[512, 0, 0], [64, 96, 200], [27, 40, 0]])
ACT = np.array([[512, 0, 0], [60, 90, 200], [27, 40, 0]])
PAR = np.array([[0, 0, 0], [12, 25, 0], [5, 0, 0]])


@pytest.mark.parametrize("dim,threads,tile,cur", [(3, 128, 2, 0), (3, 64, 8, 1), (3, 256, 1, 6),
                                                  (2, 128, 4, 3)])
def test_plan_follows_the_level_recursion(lib, dim, threads, tile, cur):
    rc, np_, phases, toff, dep = call_plan(lib, dim, MEMBER_LMAX, IDS, ACT, PAR, threads, tile, cur)
    assert rc == 0
    want = expected_phases(3, IDS, ACT, PAR, cur)
    assert np_ == len(want) == 2 ** 4 - 3          # 2^(L_max+1) - 3 with every level present
    got = [tuple(phases[4 * k:4 * k + 4]) for k in range(np_)]
    assert got == want
    n = len(MEMBER_LMAX)
    tiles = np.zeros((np_, n), np.int64)
    for k, (kind, L, _, _) in enumerate(want):
        for i in range(n):
            tiles[k, i] = member_tiles(kind, L, i, MEMBER_LMAX, ACT, PAR, dim, threads, tile)
            assert toff[k * (n + 1) + i + 1] - toff[k * (n + 1) + i] == tiles[k, i], (k, i)
        assert toff[k * (n + 1)] == 0
    for i in range(n):
        for k in range(np_):
            d = dep[k * n + i]
            dk, wrap = d >> 1, d & 1
            # the member's previous phase with tiles, scanning back cyclically
            back = next((b for b in range(1, np_ + 1) if tiles[(k - b) % np_, i] > 0), None)
            if back is None:
                continue
            assert dk == (k - back) % np_ and wrap == (1 if k - back < 0 else 0), (k, i, d)
            # progress: the tiles waited for come earlier in the queue order
            assert (wrap == 0 and dk < k) or (wrap == 1 and dk >= k)


def test_members_without_deeper_levels_wait_on_their_own_phases(lib):
    rc, np_, phases, toff, dep = call_plan(lib, 3, MEMBER_LMAX, IDS, ACT, PAR, 128, 2, 0)
    n = len(MEMBER_LMAX)
    kinds = [tuple(phases[4 * k:4 * k + 2]) for k in range(np_)]
    c0 = kinds.index((COLLIDE, 0))
    # member 0 has tiles only in the level-0 collide-stream: it waits for the
    # same phase of the previous coarse step
    assert dep[c0 * n + 0] == 2 * c0 + 1
    for k in range(np_):
        if k != c0:
            assert toff[k * (n + 1) + 1] == toff[k * (n + 1)]


def test_plan_rejects_bad_arguments(lib):
    assert call_plan(lib, 4, MEMBER_LMAX, IDS, ACT, PAR, 128, 2, 0)[0] == -1
    assert call_plan(lib, 3, MEMBER_LMAX, IDS, ACT, PAR, 96, 2, 0)[0] == -1
    assert call_plan(lib, 3, MEMBER_LMAX, IDS, ACT, PAR, 128, 9, 0)[0] == -1
    assert call_plan(lib, 3, [1, 4, 2], IDS, ACT, PAR, 128, 2, 0)[0] == -1
    assert call_plan(lib, 3, MEMBER_LMAX, IDS, ACT, PAR, 128, 2, 0, max_phases=4)[0] == -1

"""Full-size parity cases: the 2D cavity run of 2000 coarse steps (64 x 64 root
cells, D2Q9, FP64, L_max 3, the vorticity criterion every 100 steps) and one
coarse step of the 3D cavity (64^3 root cells, D3Q19, L_max 4, capacity
524,288 blocks) on a layered mesh with all four levels populated.

Shared by the GPU tests (`test_gpu_fullsize.py`) and by the script that
writes their expected values from the oracle (`golden/make_fullsize.py`).
This module defines the cases -- configurations, seeded marks, seeded states,
the sampled blocks -- and a digest of the integer mesh tables; the values
themselves come from the oracle alone."""
import hashlib

import numpy as np

import workloads as W
from oracle.lattice import equilibrium

NONE = -1

# 2D cavity, the complete run
C0_PERIODS, C0_EVERY = 20, 100
C0_SAMPLE_SEED = 77


def c0_config():
    return W.config_c0()


# 3D cavity of the headline configuration cut to 32^3 root cells (same Re,
# L_max 4), 150 coarse steps with the criterion every 50
C1CUT_PERIODS, C1CUT_EVERY = 3, 50
C1CUT_SAMPLE_SEED = 79


def c1cut_config():
    return W.config_c1(n=32, max_blocks=(32 // 4) ** 3 * 80)


# 3D cavity, one coarse step on a layered mesh
C1_SLABS = ((12.0, 0.02), (8.0, 0.02), (2.0, 0.0))   # (half width, extra fraction) per level
C1_CENTRE = 32.0
C1_MARK_SEED = 2024
C1_STATE_SEED = 31
C1_SAMPLE_SEED = 78


def c1_config():
    return W.config_c1(n=64, max_blocks=(64 // 4) ** 3 * 128)


def c1_marks(level, status, corner_z, r):
    """Marks of round r (refining leaves of level r) from the block tables."""
    half, extra = C1_SLABS[r]
    width = 4.0 / 2 ** r
    return W.slab_marks(level, status, corner_z, r, width, C1_CENTRE, half, extra,
                        C1_MARK_SEED + r)


def table_digest(level, status, child0, parent, nbr, id_sets, gaps, coords, classes):
    """SHA-256 over the block, neighbour, ID-set and gap tables, and over the
    coordinates and cell classes of the blocks in the ID sets."""
    h = hashlib.sha256()
    for a in (level, status, child0, parent, nbr):
        h.update(np.ascontiguousarray(a, np.int64).tobytes())
    for s in id_sets:
        h.update(np.asarray([len(s)] + list(s), np.int64).tobytes())
    h.update(np.asarray(gaps, np.int64).tobytes())
    act = np.sort(np.asarray([b for s in id_sets for b in s], np.int64))
    h.update(np.ascontiguousarray(np.asarray(coords, np.float64)[act]).tobytes())
    h.update(np.ascontiguousarray(np.asarray(classes)[act].astype(np.int8)).tobytes())
    return h.hexdigest()


def oracle_digest(mesh):
    cls = np.zeros((mesh.cap, mesh.m), np.int8)
    for b in mesh.active_ids():
        cls[b] = mesh.cell_classes(b)
    return table_digest(mesh.level, mesh.status, mesh.child0, mesh.parent, mesh.nbr,
                        mesh.id_sets, mesh.gap, mesh.X, cls)


def gpu_digest(gpu):
    blk = gpu.blocks()
    return table_digest(blk["level"], blk["status"], blk["child0"], blk["parent"], gpu.nbr(),
                        gpu.id_sets(), gpu.gaps(), gpu.coords(), gpu.masks())


def sample_blocks(level, status, child0, nbr, lmax, nc, seed, per_kind=4):
    """Sampled block IDs per level: leaves with a missing same-level neighbour
    (they hold ghost and interface cells), other leaves, and refined blocks
    that exchange with their children (their interface-parent cells are the
    averaged values)."""
    level, status = np.asarray(level), np.asarray(status)
    child0, nbr = np.asarray(child0), np.asarray(nbr)
    has_none = np.any(nbr == NONE, axis=1)
    exch = np.zeros(len(level), bool)
    for b in np.nonzero((status >= 2) & (child0 >= 0))[0]:
        exch[b] = bool(np.any(has_none[child0[b]:child0[b] + nc]))
    g = W.rng(seed)
    out = []
    for L in range(lmax):
        lev = level == L
        leaf = lev & (status == 1)
        for kind in (leaf & has_none, leaf & ~has_none, lev & exch):
            ids = np.nonzero(kind)[0]
            if len(ids):
                out.extend(g.choice(ids, min(per_kind, len(ids)), replace=False).tolist())
    return np.array(sorted(set(out)), np.int64)


def valid_cells(ids, status, child0, classes, dim):
    """[len(ids), 4^dim] bool: the cells of each block that carry the method's
    result.  A leaf: every cell.  A refined block: the cells over ghost or
    interface cells of its children (the coarse cells that feed interpolation
    and receive averages); cells over interior children are covered and are
    neither read nor written by the method (their values are left over)."""
    classes = np.asarray(classes)
    m = 4 ** dim
    l = np.arange(m)
    i, j, k = l % 4, (l // 4) % 4, l // 16
    child = (i >> 1) + 2 * (j >> 1) + (4 * (k >> 1) if dim == 3 else 0)
    fine = 2 * (i & 1) + 8 * (j & 1) + (32 * (k & 1) if dim == 3 else 0)
    out = np.ones((len(ids), m), bool)
    for r, b in enumerate(ids):
        if status[b] >= 2:
            out[r] = classes[child0[b] + child, fine] != 0
    return out


def seeded_state(vs, rest, id_sets, cap, m, seed, chunk=1 << 20):
    """f [cap, m, q]: the equilibrium of seeded random rho, u plus seeded noise
    on every block of the ID sets (ascending ID order), rest elsewhere."""
    act = np.sort(np.asarray([b for s in id_sets for b in s], np.int64))
    n = len(act) * m
    rho, u = W.random_macro(seed, n, vs.dim)
    noise = W.random_noise(seed + 1, (n, vs.q), 1e-3)
    f = np.empty((cap, m, vs.q))
    f[:] = rest
    flat = np.empty((n, vs.q))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        flat[s:e] = equilibrium(vs, rho[s:e], u[s:e]) + noise[s:e]
    f[act] = flat.reshape(len(act), m, vs.q)
    return f

"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the
benchmark.

This module holds workload *descriptions* (domain sizes, boundary faces,
viscosity from the Reynolds number, refinement parameters) and seeded random
number draws.  It contains none of the lattice Boltzmann or mesh-adaptation
arithmetic: the oracle and the CUDA library each implement that on their own.

Config dictionary keys
----------------------
dim, q            velocity set (2, 9) | (3, 19) | (3, 27)
nx, ny, nz        root grid in cells, multiples of 4 (nz == 4 and ignored in 2D)
max_levels        L_max >= 1
nu0               kinematic viscosity in root-lattice units
faces             2*dim entries in the order x-, x+, y-, y+, (z-, z+); each is
                  (kind, (ux, uy, uz)) with kind one of 'noslip', 'moving',
                  'outlet', 'periodic'
crit_start        N_start of the vorticity criterion
crit_inc          N_inc of the vorticity criterion
max_blocks        block capacity (IDs 0 .. max_blocks-1)
solid             None or (x0, x1, y0, y1): a square prism spanning z, in
                  root-cell units; a cell is solid when its centre lies inside
length_x          physical domain length along x (dx_0 = length_x / nx)
refine_dist       distance refinement: physical distance d_spec (0 = off)
refine_dist_targets  bit 0 the solid prism, bit 1 the outlet faces, bit 2 the wall faces
refine_dist_freeze   1: blocks refined by distance are never coarsened
"""
import numpy as np

FACE_KINDS = ("noslip", "moving", "outlet", "periodic")


def _round_capacity(max_blocks, n_root, nc):
    # keep (capacity - root blocks) a multiple of the child-group size
    cap = max(int(max_blocks), n_root + nc)
    cap += (-(cap - n_root)) % nc
    return cap


def root_blocks(cfg):
    n = (cfg["nx"] // 4) * (cfg["ny"] // 4)
    if cfg["dim"] == 3:
        n *= cfg["nz"] // 4
    return n


def finalize(cfg):
    nc = 4 if cfg["dim"] == 2 else 8
    cfg["max_blocks"] = _round_capacity(cfg["max_blocks"], root_blocks(cfg), nc)
    return cfg


def cavity(dim=2, q=None, n=64, re=100.0, u_lid=0.05, max_levels=3,
           crit_start=-2, crit_inc=1, max_blocks=None, ny=None, nz=None,
           refine_dist=0.0, refine_dist_freeze=0):
    """Lid-driven cavity (Section 5.2): all walls no-slip, the top wall (y+ in
    2D, z+ in 3D) moves along +x with speed u_lid.  nu0 = u_lid * n / Re in
    root-lattice units (characteristic length = cavity side)."""
    q = q or (9 if dim == 2 else 19)
    ny = ny or n
    nz = (nz or n) if dim == 3 else 4
    faces = [("noslip", (0.0, 0.0, 0.0)) for _ in range(2 * dim)]
    faces[2 * dim - 1] = ("moving", (u_lid, 0.0, 0.0))
    nroot = (n // 4) * (ny // 4) * ((nz // 4) if dim == 3 else 1)
    cfg = dict(dim=dim, q=q, nx=n, ny=ny, nz=nz, max_levels=max_levels,
               nu0=u_lid * n / re, faces=faces, crit_start=crit_start,
               crit_inc=crit_inc,
               max_blocks=max_blocks or nroot * 6 + 64,
               solid=None, length_x=1.0, refine_dist=refine_dist,
               refine_dist_targets=4 if refine_dist > 0 else 0,
               refine_dist_freeze=refine_dist_freeze)
    return finalize(cfg)


def periodic_box(dim=2, q=None, n=32, nu0=0.05, max_levels=1, max_blocks=None,
                 ny=None, nz=None):
    """Fully periodic box (Taylor-Green and random-field parity cases)."""
    q = q or (9 if dim == 2 else 19)
    ny = ny or n
    nz = (nz or n) if dim == 3 else 4
    faces = [("periodic", (0.0, 0.0, 0.0)) for _ in range(2 * dim)]
    nroot = (n // 4) * (ny // 4) * ((nz // 4) if dim == 3 else 1)
    cfg = dict(dim=dim, q=q, nx=n, ny=ny, nz=nz, max_levels=max_levels,
               nu0=nu0, faces=faces, crit_start=-2, crit_inc=1,
               max_blocks=max_blocks or nroot * 4 + 64, solid=None,
               length_x=1.0)
    return finalize(cfg)


def channel_cylinder(q=27, nx=256, ny=64, nz=64, side=8, cx=64, cy=32,
                     u0=0.05, re=100.0, max_levels=5, max_blocks=None,
                     crit_start=-3, crit_inc=1, refine_dist=0.15, span_periodic=False,
                     dim=3):
    """Channel past a square prism (Section 5.3): uniform inlet at x- and far
    field on the other side faces (moving-wall bounce-back with
    u = (u0, 0, 0)), anti-bounce-back outlet at x+.  nu0 = u0 * side / Re.
    Blocks within refine_dist / 2^L of the prism or the outlet are refined and
    frozen (the paper's 0.15 / 2^L rule, channel length 1).  dim = 2: the
    paper's 2D case (D2Q9 unless q is given; nz is ignored); dim = 3 spans the
    prism along z, span_periodic: periodic z faces (a quasi-2D flow when nz is
    one block)."""
    faces = [("moving", (u0, 0.0, 0.0)), ("outlet", (0.0, 0.0, 0.0)),
             ("moving", (u0, 0.0, 0.0)), ("moving", (u0, 0.0, 0.0)),
             ("moving", (u0, 0.0, 0.0)), ("moving", (u0, 0.0, 0.0))]
    if span_periodic:
        faces[4] = faces[5] = ("periodic", (0.0, 0.0, 0.0))
    if dim == 2:
        faces = faces[:4]
        q = 9
        nz = 4
    h = side / 2.0
    nroot = (nx // 4) * (ny // 4) * ((nz // 4) if dim == 3 else 1)
    cfg = dict(dim=dim, q=q, nx=nx, ny=ny, nz=nz, max_levels=max_levels,
               nu0=u0 * side / re, faces=faces, crit_start=crit_start,
               crit_inc=crit_inc, max_blocks=max_blocks or nroot * 8 + 64,
               solid=(cx - h, cx + h, cy - h, cy + h), length_x=1.0,
               refine_dist=refine_dist, refine_dist_targets=3, refine_dist_freeze=1)
    return finalize(cfg)


# --------------------------------------------------------------- seeded draws

def rng(seed):
    return np.random.default_rng(int(seed))


def random_macro(seed, n_cells, dim, drho=0.02, umax=0.04):
    """Seeded density and velocity samples: rho in 1 +- drho, |u_i| <= umax."""
    g = rng(seed)
    rho = 1.0 + drho * (2.0 * g.random(n_cells) - 1.0)
    u = umax * (2.0 * g.random((n_cells, dim)) - 1.0)
    return rho, u


def random_noise(seed, shape, scale=1e-3):
    """Seeded uniform noise in [-scale, scale)."""
    return scale * (2.0 * rng(seed).random(shape) - 1.0)


def random_marks(seed, n, p_refine=0.3, p_coarsen=0.3):
    """Seeded per-block marks: +1 refine, -1 coarsen, 0 keep (int8)."""
    x = rng(seed).random(n)
    m = np.zeros(n, dtype=np.int8)
    m[x < p_refine] = 1
    m[(x >= p_refine) & (x < p_refine + p_coarsen)] = -1
    return m


def slab_marks(level, status, corner_z, lvl, width, centre, half, p_extra, seed):
    """Seeded refinement marks for a layered mesh: every leaf (status 1) of
    level `lvl` whose block centre lies within `half` (root-cell units) of the
    plane z = centre, plus each other leaf of that level with probability
    `p_extra`.  Inputs are per-ID tables (level, status, corner z) of equal
    length; `width` is the block width of level `lvl`."""
    level, status = np.asarray(level), np.asarray(status)
    zc = np.asarray(corner_z, np.float64) + 0.5 * width
    leaf = (level == lvl) & (status == 1)
    x = rng(seed).random(len(level))
    m = np.zeros(len(level), dtype=np.int8)
    m[leaf & ((np.abs(zc - centre) < half) | (x < p_extra))] = 1
    return m


def grid_positions(shape):
    """Integer positions of the points of a grid of `shape` (2 or 3 extents)
    in x-fastest order, one row per point."""
    idx = np.arange(int(np.prod(shape)))
    pos = [idx % shape[0], (idx // shape[0]) % shape[1]]
    if len(shape) == 3:
        pos.append(idx // (shape[0] * shape[1]))
    return np.stack(pos, axis=1)


def root_positions(cfg):
    """Integer positions (bx, by[, bz]) of the root blocks in x-fastest order."""
    d = cfg["dim"]
    return grid_positions([cfg["nx"] // 4, cfg["ny"] // 4] + ([cfg["nz"] // 4] if d == 3 else []))


def morton_ids(shape):
    """IDs numbering the points of a grid (x-fastest positions) along the
    Morton (Z-order) curve: the ID of the point at position i is its rank in
    bit-interleaved order of its coordinates."""
    pos = grid_positions(shape)
    key = np.zeros(len(pos), np.int64)
    for bit in range(21):
        for ax in range(pos.shape[1]):
            key |= ((pos[:, ax] >> bit) & 1).astype(np.int64) << (bit * pos.shape[1] + ax)
    ids = np.empty(len(pos), np.int32)
    ids[np.argsort(key, kind="stable")] = np.arange(len(pos), dtype=np.int32)
    return ids


def morton_root_ids(cfg):
    """root_ids numbering the root blocks along the Morton (Z-order) curve."""
    d = cfg["dim"]
    return morton_ids([cfg["nx"] // 4, cfg["ny"] // 4] + ([cfg["nz"] // 4] if d == 3 else []))


def shuffled_root_ids(cfg, seed):
    """root_ids of a seeded random numbering of the root blocks."""
    n = len(root_positions(cfg))
    return rng(seed).permutation(n).astype(np.int32)


CELL_ARRANGEMENTS = ("calculated", "retrieved", "morton", "shuffled")


def cell_ids(shape, arrangement, seed=0):
    """Element IDs of the cells of a uniform grid (x-fastest positions) for
    the cell-based arrangements of the cell-versus-block comparison: None for
    the x-fastest numbering with computed neighbours ('calculated'), the
    identity ('retrieved': the same numbering, neighbours from a table), the
    Morton numbering, or a seeded shuffle."""
    n = int(np.prod(shape))
    if arrangement == "calculated":
        return None
    if arrangement == "retrieved":
        return np.arange(n, dtype=np.int32)
    if arrangement == "morton":
        return morton_ids(shape)
    if arrangement == "shuffled":
        return rng(seed).permutation(n).astype(np.int32)
    raise ValueError(arrangement)


# ------------------------------------------------------- named configurations

def config_c0():
    """2D lid-driven cavity, D2Q9, FP64: 64x64 root cells, Re 100, lid 0.05,
    up to 2 extra levels (L_max = 3), adapt every 100 coarse steps, 2000 steps."""
    return cavity(dim=2, q=9, n=64, re=100.0, max_levels=3, max_blocks=256 * 24)


def config_c1(n=64, re=1000.0, max_blocks=None):
    """3D lid-driven cavity, D3Q19, FP32: 64^3 root cells, Re 1000, lid 0.05,
    up to 3 extra levels (L_max = 4), adapt every 50 coarse steps."""
    nroot = (n // 4) ** 3
    return cavity(dim=3, q=19, n=n, re=re, max_levels=4,
                  max_blocks=max_blocks or nroot * 128)


def batched_cavities(n=64, seed=0):
    """Configurations of n independent 3D cavities (D3Q19) with seeded uneven
    root grids (32^3 .. 64^3 cells), depths (0 .. 3 extra levels) and Reynolds
    numbers (uniform in [100, 3200]); capacities 1, 9, 24, 48 blocks per root
    for 0, 1, 2, 3 extra levels."""
    g = rng(seed)
    sizes = g.choice([32, 40, 48, 56, 64], size=n)
    extra = g.integers(0, 4, size=n)
    res = g.uniform(100.0, 3200.0, size=n)
    out = []
    for i in range(n):
        root = (int(sizes[i]) // 4) ** 3
        cap = root * {0: 1, 1: 9, 2: 24, 3: 48}[int(extra[i])]
        out.append(cavity(dim=3, q=19, n=int(sizes[i]), re=float(res[i]),
                          max_levels=1 + int(extra[i]), max_blocks=cap))
    return out


def config_uniform_bar(n=256):
    """Single-level D3Q19 periodic block forest of n^3 cells (roofline bar)."""
    return periodic_box(dim=3, q=19, n=n, nu0=0.01, max_levels=1,
                        max_blocks=(n // 4) ** 3)

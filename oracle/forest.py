"""Block forest of quad/octrees -- Section 3.2 (data structures, ID sets, gap
set), Section 3.3 (refinement and coarsening, Algorithm 1, Algorithm 2),
Section 3.4 (ghost / interface / interior cells).  Test infrastructure only.

Plain restatement, not the paper's kernels: connectivity is rebuilt after
every adaptation by a brute-force coordinate search over all active blocks
(the geometric definition that the paper's Algorithm 2 computes by formulas).

Conventions (readings of the paper where it is silent or garbled)
-----------------------------------------------------------------
* Blocks are 4^dim cells; cell l = i + 4 j + 16 k inside a block.  Children of
  a block are N_c = 2^dim consecutive IDs; child c = cx + 2 cy + 4 cz sits at
  X_parent + (cx, cy, cz) * w_child, where w_child is half the parent block
  width (Algorithm 1 with dx_root read as the root *block* width).
  Coordinates are in root-cell units; all offsets are exact binary fractions.
* Root blocks are numbered x-fastest, b = bx + nbx (by + nby bz), unless the
  configuration gives `root_ids`: root_ids[i] is then the ID of the root at
  x-fastest position i (a relabelling only; the ID set of level 0 stays in
  ascending ID order).
* nbr[b][k] for the 3^dim directions in velocity-set order (D2Q9 / D3Q27):
  the ID of the same-level block at X_b + e_k * width, nbr[b][0] = b,
  NONE (-1) when no block of that level covers that position, or a boundary
  code -2 - face when the position leaves the domain through a wall face
  (face order x-, x+, y-, y+, z-, z+; precedence outlet > moving > no-slip,
  ties to the lowest face index).  Periodic faces wrap.
* nbr_child[b][k]: child0 of the neighbour if it exists and has children,
  the boundary code if nbr is a boundary code, else NONE.
* Refinement (Section 3.3, Section 4.4): a block may be refined if it is a leaf
  (UNREFINED), its level is below L_max - 1, and none of its neighbours is
  NONE (no same-level neighbour means a coarser block is adjacent; refining
  would break 2:1 balance -- the refinement cancel of Section 4.4).
  It may be coarsened if its status is REFINED (every child is a leaf and it
  is not REFINED_PERMANENT).
* Capacity: if the gap set holds fewer than N_c * N_refine IDs, every refine
  mark of the call is dropped (coarsening still applies); adapt() reports it.
* 2:1 enforcement (step 3): a coarsen mark is reverted when any child C has,
  in any direction k (including k = 0), a same-level neighbour N = nbr[C][k]
  that already has children or is marked for refinement in this call.
* Allocation (steps 2, 4): the refine-marked blocks, in ascending ID order,
  take groups of N_c IDs popped from the top of the gap stack; the gap stack
  is initialised in reverse so the smallest IDs come first; the first ID of
  a group is child 0.
* Removal (step 5): removed child IDs are listed by (child level, parent ID,
  child index) and appended to the gap stack in reverse, so later pops return
  them in that order; freed IDs are not reused within the same call.
* ID sets (steps 5, 6): per level, removed IDs are deleted keeping order, then
  new children are appended in (parent ID, child index) order.
* Status (step 7): refine-marked -> REFINED, applied coarsen -> UNREFINED,
  reverted coarsen -> unchanged, new -> UNREFINED, removed -> INACTIVE; then a
  refined block with at least one refined child is REFINED_WITH_CHILD,
  otherwise REFINED (REFINED_PERMANENT is kept).
* Cells (Section 3.4): the class of a cell is decided by its Chebyshev distance
  d, in cells of its own level, to the nearest position not covered by a
  same-level block (directions with nbr == NONE; walls do not count):
  d in {1, 2} ghost, d in {3, 4} interface, otherwise interior.  A refined
  block takes part in coarse-fine communication (block mask) when any of its
  children has a NONE neighbour.
"""
import numpy as np

from .lattice import velocities
from .uniform import link_face

NONE = -1
INACTIVE, UNREFINED, REFINED, REFINED_WITH_CHILD, REFINED_PERMANENT = 0, 1, 2, 3, 4
REFINED_ANY = (REFINED, REFINED_WITH_CHILD, REFINED_PERMANENT)
INTERIOR, INTERFACE, GHOST = 0, 1, 2

BLOCK_EDGE = 4


def local_coords(dim):
    """(i, j[, k]) of every cell l of a block, shape [4^dim, dim]."""
    m = BLOCK_EDGE ** dim
    l = np.arange(m)
    cols = [l % 4, (l // 4) % 4]
    if dim == 3:
        cols.append(l // 16)
    return np.stack(cols, axis=1)


class Forest:
    def __init__(self, cfg):
        self.cfg = cfg
        self.dim = d = cfg["dim"]
        self.nc = 2 ** d
        self.nk = 3 ** d
        self.m = BLOCK_EDGE ** d
        self.dirs = velocities(d, 9 if d == 2 else 27)
        self.extent = np.array([cfg["nx"], cfg["ny"], cfg["nz"]][:d], dtype=np.float64)
        self.nroot = tuple(int(e) // BLOCK_EDGE for e in self.extent)
        self.faces = cfg["faces"]
        self.lmax = cfg["max_levels"]
        self.cap = cap = cfg["max_blocks"]
        self.level = np.full(cap, -1, np.int64)
        self.X = np.zeros((cap, d), np.float64)
        self.status = np.full(cap, INACTIVE, np.int64)
        self.child0 = np.full(cap, NONE, np.int64)
        self.parent = np.full(cap, NONE, np.int64)
        self.nbr = np.full((cap, self.nk), NONE, np.int64)
        self._build_root()

    # ------------------------------------------------------------ geometry
    def width(self, level):
        return BLOCK_EDGE / (2.0 ** level)

    def _build_root(self):
        d = self.dim
        n0 = int(np.prod(self.nroot))
        self.n_root = n0
        ids = self.cfg.get("root_ids")
        ids = list(range(n0)) if ids is None else [int(v) for v in ids]
        assert sorted(ids) == list(range(n0)), "root_ids must be a permutation"
        for i in range(n0):
            b = ids[i]
            bx = i % self.nroot[0]
            by = (i // self.nroot[0]) % self.nroot[1]
            pos = [bx, by] + ([i // (self.nroot[0] * self.nroot[1])] if d == 3 else [])
            self.X[b] = np.array(pos, np.float64) * BLOCK_EDGE
            self.level[b] = 0
            self.status[b] = UNREFINED
        self.id_sets = [list(range(n0))] + [[] for _ in range(self.lmax - 1)]
        # gap set enumerated in reverse: the top of the stack (end of the
        # list) is the smallest free ID
        self.gap = list(range(self.cap - 1, n0 - 1, -1))
        self.connect()

    def active_ids(self):
        return [b for ids in self.id_sets for b in ids]

    def neighbour_position(self, b, k):
        """Position of the same-level neighbour in direction k, and the wall
        code if it leaves the domain (else None)."""
        w = self.width(self.level[b])
        pos = self.X[b] + self.dirs[k] * w
        crossed = []
        for a in range(self.dim):
            for side, outside in ((0, pos[a] < 0), (1, pos[a] >= self.extent[a])):
                if outside:
                    fi = 2 * a + side
                    if self.faces[fi][0] == "periodic":
                        pos[a] = pos[a] % self.extent[a]
                    else:
                        crossed.append(fi)
        if crossed:
            return pos, -2 - link_face(crossed, self.faces)
        return pos, None

    def connect(self):
        """Brute-force connectivity: nbr of every active block by coordinate
        lookup among the active blocks of the same level."""
        table = {}
        for b in self.active_ids():
            table[(int(self.level[b]),) + tuple(self.X[b])] = b
        self.nbr[:] = NONE
        for b in self.active_ids():
            for k in range(self.nk):
                pos, code = self.neighbour_position(b, k)
                if code is not None:
                    self.nbr[b, k] = code
                else:
                    self.nbr[b, k] = table.get((int(self.level[b]),) + tuple(pos), NONE)
        self._classes = {}
        self._lists = {}

    def nbr_child(self, b):
        out = np.full(self.nk, NONE, np.int64)
        for k in range(self.nk):
            n = self.nbr[b, k]
            if n <= -2:
                out[k] = n
            elif n >= 0 and self.child0[n] >= 0:
                out[k] = self.child0[n]
        return out

    # --------------------------------------------------------- cell classes
    def cell_classes(self, b):
        """Class (INTERIOR / INTERFACE / GHOST) of every cell of block b."""
        if b in self._classes:
            return self._classes[b]
        lc = local_coords(self.dim)
        dist = np.full(self.m, 1 << 30, np.int64)
        for k in range(1, self.nk):
            if self.nbr[b, k] != NONE:
                continue
            e = self.dirs[k]
            dk = np.zeros(self.m, np.int64)
            for a in range(self.dim):
                if e[a] < 0:
                    dk = np.maximum(dk, lc[:, a] + 1)
                elif e[a] > 0:
                    dk = np.maximum(dk, BLOCK_EDGE - lc[:, a])
            dist = np.minimum(dist, dk)
        cls = np.full(self.m, INTERIOR, np.int64)
        cls[dist <= 4] = INTERFACE
        cls[dist <= 2] = GHOST
        self._classes[b] = cls
        return cls

    def has_none(self, b):
        return bool(np.any(self.nbr[b, 1:] == NONE))

    def block_mask(self, b):
        """Coarse-fine participation of a refined block: any child with a
        NONE neighbour."""
        c0 = self.child0[b]
        if c0 < 0:
            return False
        return any(self.has_none(c0 + c) for c in range(self.nc))

    def _cached(self, key, fn):
        if key not in self._lists:
            self._lists[key] = fn()
        return self._lists[key]

    def active_list(self, level):
        """Blocks advanced on a level: leaves, and refined blocks whose block
        mask is set."""
        return self._cached(("active", level), lambda: [
            b for b in self.id_sets[level]
            if self.status[b] == UNREFINED
            or (self.status[b] in REFINED_ANY and self.block_mask(b))])

    def parent_list(self, level):
        """Refined blocks of a level that exchange data with their children."""
        return self._cached(("parent", level), lambda: [
            b for b in self.id_sets[level]
            if self.status[b] in REFINED_ANY and self.block_mask(b)])

    def boundary_children(self, level):
        """Blocks of a level with at least one NONE neighbour (they hold the
        ghost and interface cells)."""
        return self._cached(("bchild", level), lambda: [
            b for b in self.id_sets[level] if self.has_none(b)])

    # ----------------------------------------------------------- adaptation
    def can_refine(self, b):
        return (self.status[b] == UNREFINED and self.level[b] < self.lmax - 1
                and not self.has_none(b))

    def can_coarsen(self, b):
        return self.status[b] == REFINED

    def adapt(self, marks, permanent=None):
        """Apply per-block marks (+1 refine, +2 refine and freeze, -1 coarsen,
        0 keep; indexed by block ID).  A frozen (or `permanent`) refined block
        becomes REFINED_PERMANENT and is never coarsened.  Returns a dict of
        counts and the list of new children."""
        marks = np.asarray(marks)
        if permanent is None:
            permanent = marks == 2
        ids = sorted(self.active_ids())
        refine = [b for b in ids if marks[b] > 0 and self.can_refine(b)]
        coarsen = [b for b in ids if marks[b] < 0 and self.can_coarsen(b)]
        capacity_error = False
        if len(refine) * self.nc > len(self.gap):
            refine = []
            capacity_error = True
        refine_set = set(refine)
        # step 3: revert coarsening next to (new or existing) finer blocks
        kept = []
        for p in coarsen:
            violating = False
            for c in range(self.nc):
                ch = self.child0[p] + c
                for k in range(self.nk):
                    n = self.nbr[ch, k]
                    if n >= 0 and (self.child0[n] >= 0 or n in refine_set):
                        violating = True
            if not violating:
                kept.append(p)
        coarsen = kept
        # steps 2 + 4: allocation and building of new children
        new_children = []
        for p in refine:
            group = [self.gap.pop() for _ in range(self.nc)]
            assert group == list(range(group[0], group[0] + self.nc)), group
            self.child0[p] = group[0]
            lq = self.level[p] + 1
            wq = self.width(lq)
            for c, ch in enumerate(group):
                off = np.array([(c >> a) & 1 for a in range(self.dim)], np.float64)
                self.level[ch] = lq
                self.X[ch] = self.X[p] + off * wq
                self.status[ch] = UNREFINED
                self.child0[ch] = NONE
                self.parent[ch] = p
                new_children.append(ch)
        # step 4/5: removal
        removed = []
        for lev in range(self.lmax):
            for p in coarsen:
                if self.level[p] == lev:
                    removed.extend(self.child0[p] + c for c in range(self.nc))
        rem_set = set(removed)
        for ch in removed:
            self.status[ch] = INACTIVE
            self.level[ch] = -1
            self.parent[ch] = NONE
            self.child0[ch] = NONE
        for p in coarsen:
            self.child0[p] = NONE
        # steps 5 + 6: ID sets
        for lev in range(1, self.lmax):
            kept_ids = [b for b in self.id_sets[lev] if b not in rem_set]
            for p in refine:
                if self.level[p] == lev - 1:
                    kept_ids.extend(self.child0[p] + c for c in range(self.nc))
            self.id_sets[lev] = kept_ids
        self.gap.extend(reversed(removed))
        # step 7: statuses
        for p in refine:
            perm = permanent is not None and bool(permanent[p])
            self.status[p] = REFINED_PERMANENT if perm else REFINED
        for p in coarsen:
            self.status[p] = UNREFINED
        for b in self.active_ids():
            if self.status[b] in (REFINED, REFINED_WITH_CHILD):
                c0 = self.child0[b]
                any_ref = any(self.status[c0 + c] in REFINED_ANY for c in range(self.nc))
                self.status[b] = REFINED_WITH_CHILD if any_ref else REFINED
        # step 8: connectivity and cell classes
        self.connect()
        return dict(n_refined=len(refine), n_coarsened=len(coarsen),
                    capacity_error=capacity_error, new_children=new_children)

    # ------------------------------------------------------------- exports
    def counts(self):
        return [len(s) for s in self.id_sets]

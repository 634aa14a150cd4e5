"""Block-forest lattice Boltzmann solver -- Section 4 (grid advancement, streaming,
collision, refinement criterion, Algorithm 3), Section 3.4 (linear coarse-to-
fine interpolation, averaging, Dupuis-Chopard rescaling), Section 5.1 (MLUPS),
Section 5.3 (momentum exchange force).  Test infrastructure only.

State: one FP64 array f[block, cell, p] holding, for every block, its
post-streaming (pre-collision) populations at the current time of its level.

Readings of the paper (where it is silent or garbled)
-----------------------------------------------------
* Streaming is the pull form f_p(x, t+1) = f*_p(x - c_p, t) on the blocks of a
  level; the paper's in-place twist is a memory layout of the same result.
  A link whose source lies in a direction with no same-level block (NONE, at
  a coarse-fine interface) takes the cell's own f*_pbar (the value is spoiled
  by design and discarded later).  Walls and solids follow oracle.uniform.
* Level relaxation: tau_L = 1/2 + 2^L (tau_0 - 1/2) (Section 4.3).
* Rescaling (Section 3.4): the printed factor tau^F/tau^C is a ratio of
  dimensional relaxation times, tau_L * dt_L; in level lattice units
  r_cf = tau_F / (2 tau_C) (coarse to fine) and r_fc = 2 tau_C / tau_F.
* Linear interpolation: the paper's 2D formula writes a_3 y for a_3 x y and
  its 3D coefficients a_5..a_7 are mislabelled / garbled; the standard
  bilinear / trilinear polynomial over the 2^dim parent cells of the child's
  quadrant is used, child cell I at local coordinate -1/4 + I/2 (cells at
  -1/4 and 5/4 are extrapolated).
* Cubic interpolation (Section 3.4.2): the polynomial with exponents 0..3 in
  each direction through all 4^dim rescaled parent cells, on the unit
  square / cube spanned by the parent's corner cell centres (parent cell m at
  m/3); child c's cell I at -1/12 + I/6 + c_d 2/3.  The coefficients come from
  the inverted Vandermonde matrix of the 4^dim sampling points, as the paper
  describes; the same interpolant then writes the ghost cells (normal step,
  synchronisation) and every cell of new children.  The stencil spans parent
  cells over interior children, which the normal step leaves covered (the
  paper does not say what they hold): with cubic interpolation the end of
  each level step averages every parent cell whose children are not ghosts
  (the averaging of the synchronisation) instead of only those over
  interface children, so the stencil reads restricted fine data.  The printed upper limit
  of the k sum (3^(N_d - 2)) is read as 3 in 3D and as the single term k = 0
  in 2D.
* Averaging: K' = mod(l/16, 2) (the printed mod((l/16)/2, 2) is garbled); the
  sum runs over the N_c children of a parent cell.
* Normal step: interpolation writes the ghost cells of level L+1 from level L
  at time t (before level L collides); averaging writes the parent cells whose
  children are interface cells.  Pre-adapt synchronisation averages every
  parent cell whose children are not ghost cells, from the second-finest level
  up, then interpolates ghost cells from level 0 down.
* Criterion: u from the moments; first-order block-local differences,
  forward (u[i+1]-u[i]) / dx_L and backward at i = 3, no halo; dx_L =
  length_x / (nx 2^L); |w|^2 block maximum; Algorithm 3 evaluated exactly as
  |w|^2 < 4^T for T = N_start - p N_inc (p = 1 .. L_max-1, last hit wins).
  Leaves with L_des > L are marked for refinement, REFINED blocks whose own
  cells give L_des <= L are marked for coarsening.
* Distance rule (Section 4.4, used by the channel flow of Section 5.3): a leaf
  on level L whose block lies within d_spec / 2^L (physical) of a target -- the
  solid prism (Euclidean distance between the block square and the prism
  square in the x-y plane), an outlet face, or (a target the paper does not
  use) a no-slip or moving wall face -- is marked for refinement
  (+2, frozen, when refine_dist_freeze); a refined block within that distance
  loses any coarsening mark.  Distances are compared squared, in root-cell
  units, without fused operations.
* Momentum exchange (Section 5.3): the printed F = 2 dx^N_d sum f* c is read
  with the time step dt = dx of the link: F = 2 dx^(N_d - 1) sum f*_p c_p over
  links from fluid cells into solid cells, dx the physical cell size of the
  cell's level; C_D = 2 F_x / (rho_0 U_0^2 D H) with the span H in 3D.
* Solid cells always hold the rest equilibrium: they are not collided,
  streamed, interpolated into or averaged into.
"""
from fractions import Fraction

import numpy as np

from .forest import (BLOCK_EDGE, GHOST, INTERFACE, NONE, REFINED, UNREFINED,
                     Forest, local_coords)
from .lattice import CS2, VelocitySet, bgk_collide, equilibrium, moments, tau_level
from .uniform import boundary_value, face_rho_w


class ForestLBM:
    def __init__(self, cfg):
        self.cfg = cfg
        self.mesh = Forest(cfg)
        self.dim = cfg["dim"]
        self.vs = VelocitySet(cfg["dim"], cfg["q"])
        self.m = self.mesh.m
        self.lc = local_coords(self.dim)
        self.tau = [tau_level(cfg["nu0"], L) for L in range(cfg["max_levels"])]
        cap = cfg["max_blocks"]
        rest = equilibrium(self.vs, np.ones(1), np.zeros((1, self.dim)))[0]
        self.f = np.tile(rest, (cap, self.m, 1))
        self.rest = rest
        self._build_stream_maps()
        self.solid = np.zeros((cap, self.m), bool)
        self._mark_solid(range(self.mesh.n_root))

    # ---------------------------------------------------------- geometry
    def _build_stream_maps(self):
        """For each (p, cell): direction index of the block that holds x - c_p
        and the cell index inside it."""
        d, q = self.dim, self.vs.q
        dir_index = {tuple(v): i for i, v in enumerate(self.mesh.dirs)}
        self.k_src = np.zeros((q, self.m), np.int64)
        self.l_src = np.zeros((q, self.m), np.int64)
        for p in range(q):
            for l in range(self.m):
                s = self.lc[l] - self.vs.c[p]
                e = tuple(int(np.floor(v / BLOCK_EDGE)) for v in s)
                s = np.mod(s, BLOCK_EDGE)
                self.k_src[p, l] = dir_index[e]
                self.l_src[p, l] = s[0] + 4 * s[1] + (16 * s[2] if d == 3 else 0)

    def cell_centres(self, b):
        """Cell-centre coordinates (root-cell units) of block b."""
        h = self.mesh.width(self.mesh.level[b]) / BLOCK_EDGE
        return self.mesh.X[b] + (self.lc + 0.5) * h

    def _mark_solid(self, blocks):
        box = self.cfg.get("solid")
        for b in blocks:
            if box is None:
                self.solid[b] = False
                continue
            x = self.cell_centres(b)
            s = (x[:, 0] > box[0]) & (x[:, 0] < box[1]) & (x[:, 1] > box[2]) & (x[:, 1] < box[3])
            self.solid[b] = s
            self.f[b][s] = self.rest

    # ------------------------------------------------------ collide/stream
    def collide_stream(self, level):
        mesh, vs = self.mesh, self.vs
        ids = np.array(mesh.id_sets[level], np.int64)
        act = np.array(mesh.active_list(level), np.int64)
        if len(act) == 0:
            return
        rows = np.full(mesh.cap, -1, np.int64)
        rows[ids] = np.arange(len(ids))
        omega = 1.0 / self.tau[level]
        fstar, _, _ = bgk_collide(vs, self.f[ids], omega)
        fstar[self.solid[ids]] = self.f[ids][self.solid[ids]]
        f_act = self.f[act]
        _, u_act = moments(vs, f_act)
        fs_act = fstar[rows[act]]
        nbr_act = mesh.nbr[act]
        solid = self.solid
        new = np.empty_like(f_act)
        for p in range(vs.q):
            pb = vs.opp[p]
            src_blk = nbr_act[:, self.k_src[p]]               # [nA, M]
            lsrc = np.broadcast_to(self.l_src[p], src_blk.shape)
            val = np.empty(src_blk.shape)
            own_opp = fs_act[:, :, pb]
            inside = src_blk >= 0
            sb = src_blk[inside]
            ls = lsrc[inside]
            val_in = fstar[rows[sb], ls, p]
            into_solid = solid[sb, ls]
            val_in = np.where(into_solid, own_opp[inside], val_in)
            val[inside] = val_in
            none = src_blk == NONE
            val[none] = own_opp[none]
            wall = src_blk <= -2
            if np.any(wall):
                for code in np.unique(src_blk[wall]):
                    m = src_blk == code
                    face = self.cfg["faces"][-2 - code]
                    u_w = np.array(face[1][:self.dim], np.float64)
                    val[m] = boundary_value(vs, face[0], p, own_opp[m], u_act[m], u_w,
                                            face_rho_w(face))
            new[:, :, p] = val
        sol = solid[act]
        new[sol] = f_act[sol]
        self.f[act] = new

    # ------------------------------------------------- grid communication
    def _rescaled(self, f, ratio):
        """f_eq + (f - f_eq) * ratio with the cell's own rho, u (Section 3.4)."""
        rho, u = moments(self.vs, f)
        feq = equilibrium(self.vs, rho, u)
        return feq + (f - feq) * ratio

    def _interp_weights(self):
        """Polynomial interpolation of the 2^dim corner values F[a] (a = ax +
        2 ay + 4 az) at the child cells: a0 + a1 x + a2 y (+ a3 z) + cross
        terms, with x_local = -1/4 + I/2.  Returns W[cell, corner] such that
        F(x_cell) = sum_a W[cell, a] F[a]."""
        d = self.dim
        x = -0.25 + 0.5 * self.lc.astype(np.float64)           # [M, d]
        nco = 2 ** d
        W = np.zeros((self.m, nco))
        for a in range(nco):
            F = np.zeros(nco)
            F[a] = 1.0
            if d == 2:
                F00, F10, F01, F11 = F[0], F[1], F[2], F[3]
                a0, a1, a2 = F00, F10 - F00, F01 - F00
                a3 = F11 - F01 - F10 + F00
                W[:, a] = a0 + a1 * x[:, 0] + a2 * x[:, 1] + a3 * x[:, 0] * x[:, 1]
            else:
                F000, F100, F010, F110 = F[0], F[1], F[2], F[3]
                F001, F101, F011, F111 = F[4], F[5], F[6], F[7]
                a0 = F000
                a1 = F100 - F000
                a2 = F010 - F000
                a3 = F001 - F000
                a_xy = F110 - F100 - F010 + F000
                a_yz = F011 - F010 - F001 + F000
                a_xz = F101 - F100 - F001 + F000
                a_xyz = F111 - F110 - F101 - F011 + F100 + F010 + F001 - F000
                X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
                W[:, a] = (a0 + a1 * X + a2 * Y + a3 * Z + a_xy * X * Y + a_yz * Y * Z
                           + a_xz * X * Z + a_xyz * X * Y * Z)
        return W

    def _cubic_weights(self):
        """W[c][cell, V]: weight of parent cell V for cell `cell` of child c
        under cubic interpolation.  Sampling point U = (m, n[, l]) sits at
        (m/3, n/3[, l/3]); A[U, V] = x^i y^j [z^k] for V = (i, j[, k]); the
        coefficients are alpha = A^-1 F and the child value sum_V alpha_V
        x^i y^j [z^k] at x_local = -1/12 + I/6 + c_d 2/3."""
        d, m = self.dim, self.m
        lc = [[int(v) for v in row] for row in self.lc]          # (i, j, k) of V, (m, n, l) of U
        # the Vandermonde matrix is ill-conditioned (about 1e6 in 3D): it is
        # inverted in exact rational arithmetic, then the weights are rounded
        A = [[_prod(Fraction(u[a], 3) ** v[a] for a in range(d)) for v in lc] for u in lc]
        Ainv = _inverse(A)
        W = []
        for c in range(2 ** d):
            off = [(c >> ax) & 1 for ax in range(d)]
            x = [[Fraction(-1, 12) + Fraction(I[a], 6) + Fraction(2 * off[a], 3)
                  for a in range(d)] for I in lc]                # child cells
            Wc = np.empty((m, m))
            for cell in range(m):
                phi = [_prod(x[cell][a] ** v[a] for a in range(d)) for v in lc]
                for U in range(m):
                    Wc[cell, U] = float(sum(phi[V] * Ainv[V][U] for V in range(m)))
            W.append(Wc)
        return W

    def quadrant_cells(self, c):
        """Parent cell index of corner a of child quadrant c."""
        d = self.dim
        q = [(c >> ax) & 1 for ax in range(d)]
        out = []
        for a in range(2 ** d):
            o = [2 * q[ax] + ((a >> ax) & 1) for ax in range(d)]
            out.append(o[0] + 4 * o[1] + (16 * o[2] if d == 3 else 0))
        return np.array(out, np.int64)

    def interpolate(self, blocks, mode):
        """Coarse-to-fine interpolation (linear, or cubic when the
        configuration says interp = 'cubic') into `blocks` (level >= 1):
        mode 'ghost' writes ghost cells, 'all' writes every cell."""
        mesh = self.mesh
        cubic = self.cfg.get("interp", "linear") == "cubic"
        if not hasattr(self, "_W"):
            self._W = self._interp_weights()
        if cubic and not hasattr(self, "_W3"):
            if self.dim not in _CUBIC_W:
                _CUBIC_W[self.dim] = self._cubic_weights()
            self._W3 = _CUBIC_W[self.dim]
        for b in blocks:
            par = mesh.parent[b]
            lf = mesh.level[b]
            ratio = self.tau[lf] / (2.0 * self.tau[lf - 1])
            c = b - mesh.child0[par]
            if cubic:
                F = self._rescaled(self.f[par], ratio)          # [M, Q] all parent cells
                vals = self._W3[c] @ F                          # [M, Q]
            else:
                corners = self.quadrant_cells(c)
                F = self._rescaled(self.f[par][corners], ratio)    # [2^d, Q]
                vals = self._W @ F                                 # [M, Q]
            if mode == "ghost":
                sel = mesh.cell_classes(b) == GHOST
            else:
                sel = np.ones(self.m, bool)
            sel &= ~self.solid[b]
            self.f[b][sel] = vals[sel]

    def average(self, blocks, mode):
        """Fine-to-coarse averaging from `blocks` (level >= 1) into their parent
        cells: mode 'interface' for parent cells over interface children,
        'sync' for every parent cell whose children are not ghosts."""
        mesh = self.mesh
        d = self.dim
        for b in blocks:
            par = mesh.parent[b]
            lf = mesh.level[b]
            ratio = 2.0 * self.tau[lf - 1] / self.tau[lf]
            cls = mesh.cell_classes(b)
            corners = self.quadrant_cells(b - mesh.child0[par])
            Fh = self._rescaled(self.f[b], ratio)
            for a in range(2 ** d):
                kids = []
                for s in range(2 ** d):
                    o = [2 * ((a >> ax) & 1) + ((s >> ax) & 1) for ax in range(d)]
                    kids.append(o[0] + 4 * o[1] + (16 * o[2] if d == 3 else 0))
                kcls = cls[kids]
                assert np.all(kcls == kcls[0])
                if mode == "interface" and kcls[0] != INTERFACE:
                    continue
                if mode == "sync" and kcls[0] == GHOST:
                    continue
                pc = corners[a]
                if self.solid[par, pc]:
                    continue
                self.f[par, pc] = np.mean(Fh[kids], axis=0)

    # ----------------------------------------------------------- stepping
    def advance(self, level):
        mesh = self.mesh
        has_fine = level + 1 < mesh.lmax and len(mesh.id_sets[level + 1]) > 0
        if has_fine:
            ghosts = mesh.boundary_children(level + 1)
            self.interpolate(ghosts, "ghost")
        self.collide_stream(level)
        if has_fine:
            self.advance(level + 1)
            self.advance(level + 1)
            if self.cfg.get("interp", "linear") == "cubic":
                # the cubic stencil is the whole parent block: its cells over
                # interior children are averaged too
                kids = [mesh.child0[p] + c for p in mesh.parent_list(level)
                        for c in range(mesh.nc)]
                self.average(kids, "sync")
            else:
                self.average(mesh.boundary_children(level + 1), "interface")

    def step(self, n=1):
        for _ in range(n):
            self.advance(0)

    def sync(self):
        """Pre-adapt synchronisation (Section 4.4)."""
        mesh = self.mesh
        for L in range(mesh.lmax - 1, 0, -1):
            self.average(list(mesh.id_sets[L]), "sync")
        for L in range(1, mesh.lmax):
            self.interpolate(mesh.boundary_children(L), "ghost")

    # ----------------------------------------------------------- criterion
    def block_vorticity_sq(self, b):
        """Block maximum of |w|^2 in physical units (see module doc)."""
        d = self.dim
        _, u = moments(self.vs, self.f[b])
        L = self.mesh.level[b]
        dx = self.cfg["length_x"] / (self.cfg["nx"] * 2.0 ** L)
        shape = (4,) * d
        ug = [u[:, a].reshape(shape[::-1]) for a in range(d)]   # [k][j][i]

        def deriv(g, axis):
            # axis 0 = x; arrays indexed [k, j, i] (3D) or [j, i] (2D)
            ax = d - 1 - axis
            fwd = np.diff(g, axis=ax)
            last = np.take(fwd, [2], axis=ax)
            return np.concatenate([fwd, last], axis=ax) / dx

        if d == 2:
            w = deriv(ug[1], 0) - deriv(ug[0], 1)
            w2 = w * w
        else:
            wx = deriv(ug[2], 1) - deriv(ug[1], 2)
            wy = deriv(ug[0], 2) - deriv(ug[2], 0)
            wz = deriv(ug[1], 0) - deriv(ug[0], 1)
            w2 = wx * wx + wy * wy + wz * wz
        return float(np.max(w2))

    def desired_level(self, w2):
        """Algorithm 3 with eps = min(1, log2|w|) < T evaluated as w^2 < 4^T."""
        lmax = self.mesh.lmax
        ns, ni = self.cfg["crit_start"], self.cfg["crit_inc"]
        ldes = lmax - 1
        for p in range(1, lmax):
            T = ns - p * ni
            if T > 1 or w2 < 4.0 ** T:
                ldes = (lmax - 1) - p
        return ldes

    def criterion_marks(self):
        """Per-block marks from the vorticity criterion and the distance rule
        (after sync())."""
        mesh = self.mesh
        marks = np.zeros(mesh.cap, np.int8)
        w2s = {}
        for b in mesh.active_ids():
            st = mesh.status[b]
            if st not in (UNREFINED, REFINED):
                continue
            w2 = self.block_vorticity_sq(b)
            w2s[b] = w2
            ldes = self.desired_level(w2)
            L = mesh.level[b]
            if st == UNREFINED and ldes > L:
                marks[b] = 1
            elif st == REFINED and ldes <= L:
                marks[b] = -1
        if self.cfg.get("refine_dist", 0.0) > 0.0:
            freeze = bool(self.cfg.get("refine_dist_freeze", 0))
            for b in mesh.active_ids():
                if self.within_refine_distance(b):
                    if mesh.status[b] == UNREFINED:
                        marks[b] = 2 if freeze else 1
                    elif marks[b] < 0:
                        marks[b] = 0
        return marks, w2s

    def within_refine_distance(self, b):
        """Distance rule of Section 4.4 (see module doc)."""
        cfg, mesh = self.cfg, self.mesh
        L = int(mesh.level[b])
        thr = (cfg["refine_dist"] * cfg["nx"] / cfg["length_x"]) / (2.0 ** L)
        thr2 = thr * thr
        w = mesh.width(L)
        X = mesh.X[b]
        targets = int(cfg.get("refine_dist_targets", 0))
        if targets & 1 and cfg.get("solid") is not None:
            x0, x1, y0, y1 = cfg["solid"]
            dx = max(x0 - (X[0] + w), X[0] - x1, 0.0)
            dy = max(y0 - (X[1] + w), X[1] - y1, 0.0)
            if dx * dx + dy * dy < thr2:
                return True
        if targets & 6:
            kinds = (("outlet",) if targets & 2 else ()) + (("noslip", "moving") if targets & 4 else ())
            for fi, face in enumerate(cfg["faces"][:2 * self.dim]):
                if face[0] not in kinds:
                    continue
                a = fi // 2
                d = (mesh.extent[a] - (X[a] + w)) if fi % 2 else X[a]
                if d * d < thr2:
                    return True
        return False

    # ------------------------------------------------------------ adapting
    def adapt(self, marks=None):
        """Sync, criterion (unless marks are given), refine/coarsen, and
        interpolate every cell of new children from their parents."""
        self.sync()
        if marks is None:
            marks, _ = self.criterion_marks()
        res = self.mesh.adapt(marks)
        self._mark_solid(res["new_children"])
        self.interpolate(res["new_children"], "all")
        return res

    # ------------------------------------------------------------- outputs
    def macroscopic(self):
        """rho [cap, M] and u [cap, M, dim] of the current state."""
        return moments(self.vs, self.f)

    def updates_per_coarse_step(self):
        """Lattice updates of one coarse step by the MLUPS definition of
        Section 5.1: sum_L 2^L (N_L - N_{L+1} / N_c), N_L = cells on level L."""
        mesh = self.mesh
        n = [len(s) * self.m for s in mesh.id_sets] + [0]
        return sum((2 ** L) * (n[L] - n[L + 1] / mesh.nc) for L in range(mesh.lmax))

    def mea_force(self, level=None):
        """Momentum-exchange force on the solid (Section 5.3):
        F = 2 dx^(dim-1) sum over fluid leaf cells x_b and links p with x_b + c_p
        solid of f*_p c_p, dx the physical cell size of the level; computed from
        the current state (post-collision values recomputed here).  No 3D value
        is printed; pinned by the momentum balance of one periodic update (the
        fluid loses F / dx^(dim-1) in lattice units)."""
        mesh, vs = self.mesh, self.vs
        F = np.zeros(self.dim)
        blocks = [b for L in range(mesh.lmax) for b in mesh.active_list(L)
                  if mesh.status[b] == UNREFINED]
        dir_index = {tuple(v): i for i, v in enumerate(mesh.dirs)}
        for b in blocks:
            if not np.any(self.solid[b]) and not self._near_solid(b):
                continue
            L = mesh.level[b]
            dx = self.cfg["length_x"] / (self.cfg["nx"] * 2.0 ** L)
            fstar, _, _ = bgk_collide(vs, self.f[b], 1.0 / self.tau[L])
            for l in range(self.m):
                if self.solid[b, l]:
                    continue
                for p in range(1, vs.q):
                    t = self.lc[l] + vs.c[p]
                    e = tuple(int(np.floor(v / BLOCK_EDGE)) for v in t)
                    nb = mesh.nbr[b, dir_index[e]]
                    if nb < 0:
                        continue
                    tl = np.mod(t, BLOCK_EDGE)
                    li = tl[0] + 4 * tl[1] + (16 * tl[2] if self.dim == 3 else 0)
                    if self.solid[nb, li]:
                        F += 2.0 * dx ** (self.dim - 1) * fstar[l, p] * vs.cf[p]
        return F

    def _near_solid(self, b):
        for k in range(1, self.mesh.nk):
            n = self.mesh.nbr[b, k]
            if n >= 0 and np.any(self.solid[n]):
                return True
        return False


_CUBIC_W = {}   # cubic interpolation weights by dimension (exact, then rounded)


def _prod(it):
    out = Fraction(1)
    for v in it:
        out *= v
    return out


def _inverse(A):
    """Inverse of a square matrix of Fractions by Gauss-Jordan elimination."""
    n = len(A)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[n:] for row in M]

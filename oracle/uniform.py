"""Dense uniform-grid BGK lattice Boltzmann solver -- Section 2 (BGK step,
moving-wall bounce-back and anti-bounce-back boundary equations).  Test
infrastructure only.

This is the plain single-grid LBM that the block-forest oracle must reproduce
exactly when no block is refined.  Cells are cell-centred; walls lie on cell
faces (link-wise, halfway boundary conditions).

Streaming is written in pull form, f_p(x, t+1) = f*_p(x - c_p, t).  When
x - c_p lies outside the domain through a non-periodic face, population
p-bar left x towards that wall and returns as p:

* no-slip / moving wall (bounce-back with known u_w):
      f_p(x) = f*_pbar(x) - 2 w_pbar rho_w (c_pbar . u_w) / cs^2
* outlet (anti-bounce-back with known pressure, u_w = velocity of x):
      f_p(x) = -f*_pbar(x) + 2 w_p rho_w (1 + (c_pbar.u_w)^2/(2 cs^4) - u_w.u_w/(2 cs^2))

The printed anti-bounce-back equation drops the square on (c.u_w); the
standard squared form is used.  A link that leaves through several faces at
once (an edge or corner) takes the face with the highest precedence
outlet > moving wall > no-slip, ties going to the lowest face index
(x-, x+, y-, y+, z-, z+); periodic faces wrap.  A link into a solid cell is a
no-slip bounce-back (u_w = 0).
"""
import numpy as np

from .lattice import CS2, VelocitySet, bgk_collide, equilibrium

KIND_RANK = {"periodic": 0, "noslip": 1, "moving": 2, "outlet": 3}


def face_rho_w(face):
    return face[2] if len(face) > 2 else 1.0


def link_face(crossed, faces):
    """Face index that governs a link leaving through the faces in `crossed`
    (an iterable of face indices), or -1 if none of them is a wall."""
    best, best_rank = -1, 0
    for fi in sorted(crossed):
        r = KIND_RANK[faces[fi][0]]
        if r > best_rank:
            best, best_rank = fi, r
    return best


def boundary_value(vs, kind, p, fstar_opp, u_cell, u_w, rho_w):
    """Value of f_p at a cell whose link p comes from a wall (see module doc).
    fstar_opp = f*_pbar(x); u_cell = velocity of x (for the outlet)."""
    c = vs.cf[p]
    w = vs.w[p]
    if kind in ("noslip", "moving"):
        cu = -(u_w @ c) if np.ndim(u_w) > 1 else -float(np.dot(c, u_w))
        return fstar_opp - 2.0 * w * rho_w * cu / CS2
    if kind == "outlet":
        cu = u_cell @ (-c)
        uu = np.sum(u_cell * u_cell, axis=-1)
        return -fstar_opp + 2.0 * w * rho_w * (1.0 + cu * cu / (2.0 * CS2 * CS2)
                                                - uu / (2.0 * CS2))
    raise ValueError(kind)


class UniformLBM:
    """Uniform grid of shape (nx, ny[, nz]) with populations f[..., Q]."""

    def __init__(self, dim, q, shape, tau, faces, solid=None):
        self.vs = VelocitySet(dim, q)
        self.dim = dim
        self.shape = tuple(shape)
        self.omega = 1.0 / tau
        self.faces = faces
        self.solid = np.zeros(self.shape, bool) if solid is None else solid
        self.f = equilibrium(self.vs, np.ones(self.shape), np.zeros(self.shape + (dim,)))
        self._build_maps()

    def _build_maps(self):
        """For every direction p: source index of every cell, and the wall face
        index (or -1) that replaces the source when it lies outside."""
        idx = np.indices(self.shape)
        self.src, self.face = [], []
        for p in range(self.vs.q):
            s = [idx[a] - self.vs.c[p, a] for a in range(self.dim)]
            face = -np.ones(self.shape, np.int64)
            rank = np.zeros(self.shape, np.int64)
            for a in range(self.dim):
                n = self.shape[a]
                for side, mask in ((0, s[a] < 0), (1, s[a] >= n)):
                    fi = 2 * a + side
                    kind = self.faces[fi][0]
                    if kind == "periodic":
                        continue
                    r = KIND_RANK[kind]
                    upd = mask & (r > rank)
                    face[upd] = fi
                    rank[upd] = r
                s[a] = np.mod(s[a], n)
            self.src.append(tuple(s))
            self.face.append(face)

    def moments(self):
        from .lattice import moments
        return moments(self.vs, self.f)

    def step(self):
        vs = self.vs
        fstar, rho, u = bgk_collide(vs, self.f, self.omega)
        fstar[self.solid] = self.f[self.solid]
        new = np.empty_like(self.f)
        for p in range(vs.q):
            pb = vs.opp[p]
            val = fstar[self.src[p] + (p,)]
            # a source inside a solid: no-slip bounce-back
            into_solid = self.solid[self.src[p]]
            val = np.where(into_solid, fstar[..., pb], val)
            face = self.face[p]
            for fi in np.unique(face[face >= 0]):
                m = face == fi
                kind, u_w = self.faces[fi][0], np.array(self.faces[fi][1][:self.dim])
                val[m] = boundary_value(vs, kind, p, fstar[..., pb][m], u[m], u_w,
                                        face_rho_w(self.faces[fi]))
            new[..., p] = val
        new[self.solid] = self.f[self.solid]
        self.f = new

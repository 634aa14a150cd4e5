"""Per-cell field comparison for the GPU parity tests.

A relative L2 norm over a whole forest dilutes an error confined to the thin
layers that interpolation, averaging and boundary links touch.  This helper
takes the worst cell instead: for every cell, max over p of
|f_gpu - f_ref| / max(|f_ref|, w_p), grouped by the cell's class (ghost,
interface, interior; Section 3.4) so that a failure names the layer it is in.
"""
import numpy as np

# per-cell bars next to the relative-L2 bars (1e-12 FP64, 1e-5 FP32)
CELL_TOL = {"f64": 1e-10, "f32": 1e-4}
CLASS_NAMES = ("interior", "interface", "ghost")


def cell_errors(got, want, classes, w, valid=None):
    """got, want: [n, M, Q]; classes: [n, M] (0 interior, 1 interface,
    2 ghost); w: [Q] weights; valid: optional [n, M] bool (cells compared).
    Returns {class name: (worst error, (row, cell)) or None}."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.maximum(np.abs(want), np.asarray(w, np.float64)[None, None, :])
    err = np.max(np.abs(got - want) / scale, axis=2)           # [n, M]
    classes = np.asarray(classes)
    if valid is None:
        valid = np.ones(err.shape, bool)
    out = {}
    for c, name in enumerate(CLASS_NAMES):
        sel = valid & (classes == c)
        if not np.any(sel):
            out[name] = None
            continue
        e = np.where(sel, err, -1.0)
        r, l = np.unravel_index(int(np.argmax(e)), e.shape)
        out[name] = (float(e[r, l]), (int(r), int(l)))
    return out


def assert_cells(got, want, classes, w, storage, valid=None, what=""):
    """Every class within CELL_TOL[storage]; the message lists all classes."""
    res = cell_errors(got, want, classes, w, valid)
    tol = CELL_TOL[storage]
    bad = {k: v for k, v in res.items() if v is not None and not v[0] <= tol}
    assert not bad, "%s per-cell error above %g: %s (all: %s)" % (what, tol, bad, res)
    return res


def oracle_classes(mesh, ids):
    """[len(ids), M] cell classes of the oracle's forest."""
    return np.stack([mesh.cell_classes(b) for b in ids])

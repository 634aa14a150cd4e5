"""The allocation-free mass audit (amr_mass_audit_noalloc) through the C ABI.

amr_mass_audit_noalloc serves callers that cannot allocate device memory: it
takes only caller-owned input and output pointers and keeps its partial sums
in a static device array of the library.  This test builds the caller-owned
inputs itself, independently of any instance's arena: the populations of an
AMR instance (exported with amr_fields) are written into the library's
stored form (block-major buffers [B][Q][M]; each pre-collision f_p(x) in the
slot of the cell x - c_p of the same level, or in x's own opposite slot
where x - c_p is not a cell of that level; 16-bit storages hold value - w_p)
in two separate buffers with the unused entries of each filled with NaN, and
a per-level buffer choice selects them.  The audit must equal an FP64 numpy sum of the same values
over the leaf cells, and the instance's own audit (AMR_MASS), on two calls
in a row with different states and buffer choices, within the FP64
tolerance of the parity tests.  D3Q19 in FP64, FP32, BF16 and FP16 storage,
and D2Q9 in FP64 (three outputs; the fourth output entry stays untouched).
It is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle.lattice import VelocitySet, equilibrium, velocities

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
STORAGE_CODE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
TORCH_DTYPE = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
               "f16": torch.float16}
SENTINEL = 12345.0


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    from paper_2308_08085_gb300.amr import load_library
    return load_library(b.build())


def instance(dim, storage):
    from paper_2308_08085_gb300 import AmrLBM
    if dim == 3:
        cfg = W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 30)
        first = [1, 5, 6]
    else:
        cfg = W.cavity(dim=2, q=9, n=16, max_levels=3, max_blocks=16 * 20)
        first = [5, 6, 9]
    sim = AmrLBM(cfg, storage=storage)
    for ids in (first, None):
        marks = np.zeros(cfg["max_blocks"], np.int8)
        if ids is None:               # refine the first child of the first parent again
            blk = sim.blocks()
            ids = [int(blk["child0"][first[0]])]
        marks[ids] = 1
        sim.adapt(torch.from_numpy(marks).cuda())
    vs = VelocitySet(dim, cfg["q"])
    n = cfg["max_blocks"] * vs_cells(dim)
    rho, u = W.random_macro(77, n, dim)
    f = equilibrium(vs, rho, u) + W.random_noise(78, (n, cfg["q"]), 1e-3)
    sim.set_populations(f.reshape(cfg["max_blocks"], vs_cells(dim), cfg["q"]))
    return sim, vs


def vs_cells(dim):
    return 4 ** dim


def stored_form(f, nbr, level, vs):
    """g [Q, B, M]: the slot of every pre-collision value f[b, l, p] in the
    library's stored form (see the module doc); NaN where nothing is stored."""
    dim, q = vs.dim, vs.q
    B, M, _ = f.shape
    dirs = velocities(dim, 9 if dim == 2 else 27)
    k_of = {tuple(int(v) for v in d): k for k, d in enumerate(dirs)}
    lc = np.stack([np.arange(M) % 4, (np.arange(M) // 4) % 4] +
                  ([np.arange(M) // 16] if dim == 3 else []), 1)
    g = np.full((q, B, M), np.nan)
    act = np.nonzero(level >= 0)[0]
    for p in range(q):
        src = lc - vs.c[p]
        off = np.floor_divide(src, 4)
        cell = np.mod(src, 4)
        cell_idx = cell[:, 0] + 4 * cell[:, 1] + (16 * cell[:, 2] if dim == 3 else 0)
        for l in range(M):
            k = k_of[tuple(int(v) for v in off[l])]
            sb = act if k == 0 else nbr[act, k]
            ok = sb >= 0
            g[p, sb[ok], cell_idx[l]] = f[act[ok], l, p]
            g[vs.opp[p], act[~ok], l] = f[act[~ok], l, p]
    return g


def encode(g, vs, storage):
    """Device tensor of the stored values in `storage`, in the library's
    block-major buffer order [B][Q][M], and the values it decodes to, [Q][B][M]
    (16-bit storages hold value - w_p; the library decodes them in FP32,
    value = float(h) + float(w_p), and sums in FP64)."""
    w = vs.w[:, None, None]
    if storage in ("bf16", "f16"):
        t = torch.from_numpy(g - w).to(TORCH_DTYPE[storage])
        dec = (t.to(torch.float32).numpy() + w.astype(np.float32)).astype(np.float64)
    else:
        t = torch.from_numpy(g).to(TORCH_DTYPE[storage])
        dec = t.to(torch.float64).numpy()
    return t.permute(1, 0, 2).contiguous().cuda(), dec


def leaf_sums(dec, nbr, level, status, vs):
    """FP64 sum over leaf cells of rho V and rho u V from the stored values
    (gathered back by the same slot rule)."""
    dim, q = vs.dim, vs.q
    _, B, M = dec.shape
    dirs = velocities(dim, 9 if dim == 2 else 27)
    k_of = {tuple(int(v) for v in d): k for k, d in enumerate(dirs)}
    lc = np.stack([np.arange(M) % 4, (np.arange(M) // 4) % 4] +
                  ([np.arange(M) // 16] if dim == 3 else []), 1)
    leaves = np.nonzero(status == 1)[0]
    f = np.zeros((len(leaves), M, q))
    for p in range(q):
        src = lc - vs.c[p]
        off = np.floor_divide(src, 4)
        cell = np.mod(src, 4)
        cell_idx = cell[:, 0] + 4 * cell[:, 1] + (16 * cell[:, 2] if dim == 3 else 0)
        for l in range(M):
            k = k_of[tuple(int(v) for v in off[l])]
            sb = leaves if k == 0 else nbr[leaves, k]
            ok = sb >= 0
            f[ok, l, p] = dec[p, sb[ok], cell_idx[l]]
            f[~ok, l, p] = dec[vs.opp[p], leaves[~ok], l]
    vol = 2.0 ** (-dim * level[leaves].astype(np.float64))
    rho = f.sum(2)
    out = [float((rho.sum(1) * vol).sum())]
    for a in range(dim):
        out.append(float(((f @ vs.cf[:, a]).sum(1) * vol).sum()))
    return np.array(out)


def audit(lib, sim, vs, storage, fa, fb, cur, nbr32, level_t, status_t, out):
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.amr_mass_audit_noalloc(vs.dim, vs.q, STORAGE_CODE[storage], sim.cap,
                                    fa.data_ptr(), fb.data_ptr(), cur, level_t.data_ptr(),
                                    status_t.data_ptr(), nbr32.data_ptr(), None,
                                    out.data_ptr(), stream)
    assert rc == 0, lib.amr_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dim,storage", [(3, "f64"), (3, "f32"), (3, "bf16"), (3, "f16"),
                                         (2, "f64")])
def test_noalloc_audit_on_two_calls(lib, dim, storage):
    sim, vs = instance(dim, storage)
    out = torch.full((4,), SENTINEL, dtype=torch.float64, device="cuda")
    for call in range(2):
        f = sim.populations()                         # [B, M, Q], pre-collision, FP64
        blk = sim.blocks()
        level, status = blk["level"], blk["status"]
        nbr = sim.nbr().astype(np.int64)              # [B, 3^dim]
        nbr32 = np.full((sim.cap, 32), -1, np.int32)
        nbr32[:, :nbr.shape[1]] = nbr
        g = stored_form(f, nbr, level, vs)
        t, dec = encode(np.nan_to_num(g, nan=0.0), vs, storage)
        # the buffer each level reads: all of B on the first call, levels
        # 0 and 2 from B and level 1 from A on the second
        cur = 0xFFFFFFFF if call == 0 else 0b101
        nan = torch.full_like(t, float("nan"))
        lev = torch.from_numpy(level).cuda()
        from_b = (((cur >> lev.clamp(min=0)) & 1) == 1)[:, None, None]
        fb = torch.where(from_b, t, nan).contiguous()
        fa = torch.where(from_b, nan, t).contiguous()
        level_t = torch.from_numpy(level.astype(np.int32)).cuda()
        status_t = torch.from_numpy(status.astype(np.int32)).cuda()
        nbr_t = torch.from_numpy(nbr32).cuda()
        got = audit(lib, sim, vs, storage, fa, fb, cur, nbr_t, level_t, status_t, out)
        want = leaf_sums(dec, nbr, level, status, vs)
        n = 1 + dim
        err = np.abs(got[:n] - want) / np.maximum(1.0, np.abs(want))
        assert np.all(err <= TOL), (call, got, want)
        if dim == 2:
            assert got[3] == SENTINEL                 # only 1 + dim outputs are written
        inst = sim.mass()[:n]
        tol_inst = TOL if storage in ("f64", "f32") else 1e-5    # 16-bit: rounding paths differ
        err = np.abs(got[:n] - inst) / np.maximum(1.0, np.abs(inst))
        assert np.all(err <= tol_inst), (call, got, inst)
        sim.step(2)                                   # a different state for the next call
    sim.close()


def test_noalloc_audit_rejects_oversize_input(lib):
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    too_many = 64 * 16384 + 1
    rc = lib.amr_mass_audit_noalloc(3, 19, 1, too_many, dummy.data_ptr(), dummy.data_ptr(), 0,
                                    dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None,
                                    out.data_ptr(), None)
    assert rc == -1
    assert b"static scratch limit" in lib.amr_last_error()

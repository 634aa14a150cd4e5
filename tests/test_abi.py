"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol declared in include/amr.h, and rejects bad configurations on the host
(no GPU call is made)."""
import ctypes
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "amr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_08085_gb300 import build as b
    from paper_2308_08085_gb300.amr import load_library
    return load_library(b.build())


def test_header_declares_abi():
    syms = declared_symbols()
    for s in ["amr_init", "amr_step", "amr_adapt", "amr_fields", "amr_free", "amr_arena_bytes",
              "amr_set_fields", "amr_strerror"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_config_struct_layout_matches_header(lib):
    from paper_2308_08085_gb300.amr import AmrAdaptStats, AmrConfig, AmrKernelProfile
    assert ctypes.sizeof(AmrConfig) == 376
    assert ctypes.sizeof(AmrAdaptStats) == 56
    assert ctypes.sizeof(AmrKernelProfile) == 64


def test_arena_bytes_and_validation(lib):
    from paper_2308_08085_gb300.amr import make_config
    cfg = W.cavity(dim=3, q=19, n=16, max_levels=3)
    c = make_config(cfg, "f32")
    n = lib.amr_arena_bytes(ctypes.byref(c))
    pops = 2 * cfg["max_blocks"] * 64 * 19 * 4
    assert n >= pops and n < pops * 3 + (64 << 20)
    # invalid: extents not a multiple of 4
    bad = make_config(dict(cfg, nx=18), "f32")
    assert lib.amr_arena_bytes(ctypes.byref(bad)) == 0
    assert b"multiples of 4" in lib.amr_last_error()
    # invalid: 16-bit storage in 2D
    bad = make_config(W.cavity(dim=2, n=16), "bf16")
    assert lib.amr_arena_bytes(ctypes.byref(bad)) == 0
    # invalid: unpaired periodic face
    cfg2 = W.periodic_box(dim=2, n=16)
    cfg2["faces"][1] = ("noslip", (0, 0, 0))
    assert lib.amr_arena_bytes(ctypes.byref(make_config(cfg2))) == 0
    # capacity not aligned to child groups
    cfg3 = W.cavity(dim=2, n=16)
    cfg3["max_blocks"] += 1
    assert lib.amr_arena_bytes(ctypes.byref(make_config(cfg3, "f64"))) == 0


def test_init_rejects_small_arena_without_gpu(lib):
    from paper_2308_08085_gb300.amr import AMR_E_ARENA, make_config
    c = make_config(W.cavity(dim=2, n=16), "f64")
    h = ctypes.c_void_p()
    rc = lib.amr_init(ctypes.byref(c), ctypes.c_void_p(256), 1024, None, ctypes.byref(h))
    assert rc == AMR_E_ARENA and not h.value


# ------------------------------------------------ cell-based uniform solver
def brute_force_cell_table(vs, shape, ids):
    """table[p][id of position i] = id of the position one link c_p downstream
    of i, periodic, by direct coordinate arithmetic."""
    import numpy as np
    pos = W.grid_positions(shape)
    n = len(pos)
    ids = np.arange(n) if ids is None else ids
    stride = [1, shape[0], shape[0] * shape[1]]
    out = np.full((vs.q, n), -1, np.int64)
    for p in range(vs.q):
        tgt = (pos + vs.c[p][:len(shape)]) % np.array(shape)
        j = sum(tgt[:, a] * stride[a] for a in range(len(shape)))
        out[p, ids] = ids[j]
    return out


@pytest.mark.parametrize("dim,q,shape", [(2, 9, [6, 5]), (3, 19, [4, 3, 5]), (3, 27, [3, 4, 2])])
@pytest.mark.parametrize("arrangement", W.CELL_ARRANGEMENTS)
def test_cells_table_matches_geometry(lib, dim, q, shape, arrangement):
    import numpy as np
    from oracle.lattice import VelocitySet
    from paper_2308_08085_gb300.amr import cells_table
    ids = W.cell_ids(shape, arrangement, seed=3)
    got = cells_table(dim, q, shape, ids)
    want = brute_force_cell_table(VelocitySet(dim, q), shape, ids)
    assert np.array_equal(got, want)
    # every row is a permutation (push streaming writes each slot once)
    assert all(np.array_equal(np.sort(r), np.arange(got.shape[1])) for r in got)


def test_cells_rejects_bad_input_without_gpu(lib):
    import numpy as np
    from paper_2308_08085_gb300.amr import AMR_E_INVAL
    n = 4 * 4
    table = np.empty(9 * n, np.int32)
    dup = np.arange(n, dtype=np.int32)
    dup[3] = 2
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.amr_cells_table(2, 9, 4, 4, 1, vp(dup), vp(table)) == AMR_E_INVAL
    assert b"permutation" in lib.amr_last_error()
    out_of_range = np.arange(n, dtype=np.int32)
    out_of_range[0] = n
    assert lib.amr_cells_table(2, 9, 4, 4, 1, vp(out_of_range), vp(table)) == AMR_E_INVAL
    assert lib.amr_cells_table(3, 15, 4, 4, 4, None, vp(table)) == AMR_E_INVAL
    assert lib.amr_cells_table(2, 9, 0, 4, 1, None, vp(table)) == AMR_E_INVAL
    buf = ctypes.c_void_p(4096)     # never dereferenced: every call below is rejected first
    assert lib.amr_cells_step(2, 9, 4, 4, 1, 7, 0.1, None, buf, ctypes.c_void_p(8192), 1,
                              None) == AMR_E_INVAL
    assert lib.amr_cells_step(2, 9, 4, 4, 1, 0, 0.1, None, buf, buf, 1, None) == AMR_E_INVAL
    assert lib.amr_cells_step(2, 9, 4, 4, 1, 1, 0.1, None, buf, ctypes.c_void_p(8192), 1,
                              None) == AMR_E_INVAL
    assert lib.amr_cells_step(2, 9, 4, 4, 1, 0, 0.0, None, buf, ctypes.c_void_p(8192), 1,
                              None) == AMR_E_INVAL


def test_root_ids_and_interp_validated_on_host(lib):
    import numpy as np
    from paper_2308_08085_gb300.amr import AMR_E_INVAL, make_config
    cfg = W.cavity(dim=2, n=16)
    for bad in ([0, 1, 2, 2] + list(range(4, 16)), [16] + list(range(1, 16)),
                [-1] + list(range(1, 16))):
        cfg["root_ids"] = np.array(bad, np.int32)
        c = make_config(cfg)
        assert lib.amr_arena_bytes(ctypes.byref(c)) == 0
        assert b"permutation" in lib.amr_last_error()
        h = ctypes.c_void_p()
        assert lib.amr_init(ctypes.byref(c), ctypes.c_void_p(256), 1 << 40, None,
                            ctypes.byref(h)) == AMR_E_INVAL and not h.value
    cfg["root_ids"] = W.shuffled_root_ids(cfg, 1)
    assert lib.amr_arena_bytes(ctypes.byref(make_config(cfg))) > 0
    c = make_config(W.cavity(dim=3, q=19, n=16))
    for interp, ok in ((0, True), (3, True), (1, False), (2, False), (-1, False)):
        c.interp = interp
        assert (lib.amr_arena_bytes(ctypes.byref(c)) > 0) == ok, interp


def test_batch_and_table_calls_reject_bad_arguments_on_the_host(lib):
    """Argument checks that return before any device call."""
    from paper_2308_08085_gb300.amr import AmrBatchConfig
    assert ctypes.sizeof(AmrBatchConfig) == 16
    out = (ctypes.c_int64 * 3)()
    ptr = ctypes.c_void_p(16)                     # never dereferenced: rejected first
    # dimension 5, a zero capacity, missing tables
    assert lib.amr_validate_tables(5, 3, 64, ptr, ptr, ptr, ptr, ptr, None, 0, out, None) == -1
    assert lib.amr_validate_tables(3, 3, 0, ptr, ptr, ptr, ptr, ptr, None, 0, out, None) == -1
    assert lib.amr_validate_tables(3, 3, 64, None, ptr, ptr, ptr, ptr, None, 0, out, None) == -1
    assert lib.amr_validate_tables(3, 3, 64, ptr, ptr, ptr, ptr, ptr, None, 4, out, None) == -1
    assert lib.amr_check_tables(None, out) == -1
    cfg = AmrBatchConfig(1, 128, 2, 0)
    assert lib.amr_batch_configure(None, ctypes.byref(cfg)) == -1
    assert lib.amr_batch_get_config(None, ctypes.byref(cfg)) == -1
    assert lib.amr_batch_step(None, 1) == -1
    assert lib.amr_batch_sync(None) == -1
    assert lib.amr_batch_check_timeout(None, 1 << 20) == -1
    assert lib.amr_batch_autotune(None, 1, 7, None, None) == -1

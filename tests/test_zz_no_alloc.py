"""The allocation-free mass audit (amr_mass_audit_noalloc) against the
instance's own audit (amr_fields with AMR_MASS).

amr_mass_audit_noalloc serves callers that cannot allocate device memory:
it takes only caller-owned input and output pointers and keeps its partial
sums in a static device array of the library.  This test feeds it the
population and block tables of an AMR instance (exported to caller-owned
device tensors) and checks, on two calls in a row with different states, that
it returns the same FP64 sums as the instance's audit within the FP64 field
tolerance of the parity tests.  It is collected last so that a run stopping
at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle.lattice import VelocitySet, equilibrium

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
STORAGE_CODE = {"f64": 0, "f32": 1}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    from paper_2308_08085_gb300.amr import load_library
    lib = load_library(b.build())
    lib.amr_mass_audit_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
    lib.amr_mass_audit_noalloc.restype = ctypes.c_int
    return lib


def instance(storage):
    from paper_2308_08085_gb300 import AmrLBM
    cfg = W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 30)
    sim = AmrLBM(cfg, storage=storage)
    marks = np.zeros(cfg["max_blocks"], np.int8)
    marks[[1, 5, 6]] = 1
    sim.adapt(torch.from_numpy(marks).cuda())
    vs = VelocitySet(3, 19)
    n = cfg["max_blocks"] * 64
    rho, u = W.random_macro(77, n, 3)
    f = equilibrium(vs, rho, u) + W.random_noise(78, (n, 19), 1e-3)
    sim.set_populations(f.reshape(cfg["max_blocks"], 64, 19))
    return sim


def audit_noalloc(lib, sim, storage, out):
    """Export the state to caller-owned device tensors and audit them."""
    from paper_2308_08085_gb300.amr import AMR_BLOCKS, AMR_F
    f = sim.fields_device(AMR_F, torch.float64)
    f = f.to(torch.float64 if storage == "f64" else torch.float32).contiguous()
    blocks = sim.fields_device(AMR_BLOCKS, torch.int32).reshape(4, sim.cap)
    level = blocks[0].contiguous()
    status = blocks[1].contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.amr_mass_audit_noalloc(3, 19, STORAGE_CODE[storage], sim.cap, f.data_ptr(),
                                    f.data_ptr(), 0, level.data_ptr(), status.data_ptr(),
                                    out.data_ptr(), stream)
    assert rc == 0, lib.amr_last_error()
    torch.cuda.synchronize()
    return out[:4].cpu().numpy()


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_noalloc_audit_matches_instance_audit_twice(lib, storage):
    sim = instance(storage)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        want = sim.mass()
        got = audit_noalloc(lib, sim, storage, out)
        err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
        assert np.all(err <= TOL), (call, got, want)
        sim.step(2)                  # a different state for the second call
    sim.close()


def test_noalloc_audit_rejects_oversize_input(lib):
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    too_many = 64 * 16384 + 1
    rc = lib.amr_mass_audit_noalloc(3, 19, 1, too_many, dummy.data_ptr(), dummy.data_ptr(), 0,
                                    dummy.data_ptr(), dummy.data_ptr(), out.data_ptr(), None)
    assert rc == -1
    assert b"static scratch limit" in lib.amr_last_error()

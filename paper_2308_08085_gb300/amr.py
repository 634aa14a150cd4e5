"""ctypes binding of the C ABI declared in include/amr.h.

Argument marshalling only: every step of the method runs in the CUDA library
libamr.so.  PyTorch provides the device arena and the stream.  If the library
has not been built the binding raises; there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libamr.so")

# status codes
AMR_OK, AMR_E_INVAL, AMR_E_CAPACITY, AMR_E_CUDA, AMR_E_TIMEOUT, AMR_E_UNSTABLE, AMR_E_ARENA = (
    0, -1, -2, -3, -4, -5, -6)
# storage
STORAGE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
# face kinds
FACE = {"noslip": 0, "moving": 1, "outlet": 2, "periodic": 3}
# field selectors
AMR_RHO_U, AMR_F, AMR_BLOCKS, AMR_COORDS, AMR_NBR, AMR_NBR_CHILD, AMR_IDSETS, AMR_GAPS, \
    AMR_MASKS, AMR_COUNTS, AMR_MASS, AMR_FORCE, AMR_FEATURES = range(13)
MLP_INPUTS, MLP_HIDDEN = 27, 64
# connectivity of the cell-based uniform solver
AMR_CELLS_CALCULATED, AMR_CELLS_RETRIEVED = 0, 1

EXPORTED = ["amr_arena_bytes", "amr_init", "amr_step", "amr_adapt", "amr_fields",
            "amr_set_fields", "amr_profile", "amr_profile_read", "amr_free", "amr_strerror",
            "amr_last_error"]


class AmrFace(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("u", ctypes.c_double * 3), ("rho_w", ctypes.c_double)]


class AmrConfig(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("q", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("crit_start", ctypes.c_int32),
                ("crit_inc", ctypes.c_int32), ("has_solid", ctypes.c_int32),
                ("max_blocks", ctypes.c_int64), ("nu0", ctypes.c_double),
                ("length_x", ctypes.c_double), ("solid", ctypes.c_double * 4),
                ("faces", AmrFace * 6), ("use_graphs", ctypes.c_int32),
                ("kernel_variant", ctypes.c_int32), ("refine_dist", ctypes.c_double),
                ("refine_dist_targets", ctypes.c_int32), ("refine_dist_freeze", ctypes.c_int32),
                ("root_ids", ctypes.POINTER(ctypes.c_int32)), ("interp", ctypes.c_int32),
                ("check_tables", ctypes.c_int32)]


class AmrAdaptStats(ctypes.Structure):
    _fields_ = [("n_marked_refine", ctypes.c_int64), ("n_marked_coarsen", ctypes.c_int64),
                ("n_refined", ctypes.c_int64), ("n_coarsened", ctypes.c_int64),
                ("n_blocks", ctypes.c_int64), ("capacity_error", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("ms_total", ctypes.c_double)]


class AmrMlpState(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("adam_m", ctypes.c_void_p),
                ("adam_v", ctypes.c_void_p), ("params_half", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("loss", ctypes.c_void_p), ("step", ctypes.c_int64)]


class AmrKernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("cells", ctypes.c_double)]


_lib = None


def validate_tables(dim, max_levels, level, status, child0, parent, nbr, gap=None,
                    stream=None):
    """amr_validate_tables on device int32 tensors (nbr [cap, 32]); returns
    (bad entries, first bad block or -1, AMR_CHECK_* code)."""
    import torch
    lib = load_library()
    cap = level.numel()
    out = (ctypes.c_int64 * 3)()
    s = stream if stream is not None else torch.cuda.current_stream(level.device)
    rc = lib.amr_validate_tables(int(dim), int(max_levels), cap, level.data_ptr(),
                                 status.data_ptr(), child0.data_ptr(), parent.data_ptr(),
                                 nbr.data_ptr(), gap.data_ptr() if gap is not None else None,
                                 gap.numel() if gap is not None else 0, out,
                                 ctypes.c_void_p(s.cuda_stream))
    if rc != AMR_OK:
        raise AmrError(rc, "amr_validate_tables")
    return tuple(int(v) for v in out)


def load_library(path=LIB_PATH):
    """Load libamr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libamr.so is not built (%s): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    lib.amr_arena_bytes.argtypes = [ctypes.POINTER(AmrConfig)]
    lib.amr_arena_bytes.restype = sz
    lib.amr_init.argtypes = [ctypes.POINTER(AmrConfig), vp, sz, vp, ctypes.POINTER(vp)]
    lib.amr_init.restype = i32
    lib.amr_step.argtypes = [vp, i32]
    lib.amr_step.restype = i32
    lib.amr_adapt.argtypes = [vp, vp, ctypes.POINTER(AmrAdaptStats)]
    lib.amr_adapt.restype = i32
    lib.amr_fields.argtypes = [vp, i32, vp, sz, i32]
    lib.amr_fields.restype = i64
    lib.amr_set_fields.argtypes = [vp, i32, vp, sz, i32]
    lib.amr_set_fields.restype = i32
    lib.amr_profile.argtypes = [vp, i32]
    lib.amr_profile.restype = i32
    lib.amr_profile_read.argtypes = [vp, ctypes.POINTER(AmrKernelProfile), i32, i32]
    lib.amr_profile_read.restype = i32
    lib.amr_free.argtypes = [vp]
    lib.amr_free.restype = i32
    lib.amr_checkpoint_bytes.argtypes = [vp]
    lib.amr_checkpoint_bytes.restype = i64
    lib.amr_checkpoint.argtypes = [vp, vp, sz]
    lib.amr_checkpoint.restype = i32
    lib.amr_restore.argtypes = [vp, vp, sz]
    lib.amr_restore.restype = i32
    lib.amr_strerror.argtypes = [i32]
    lib.amr_strerror.restype = ctypes.c_char_p
    lib.amr_last_error.argtypes = []
    lib.amr_last_error.restype = ctypes.c_char_p
    lib.amr_mlp_param_count.argtypes = []
    lib.amr_mlp_param_count.restype = i32
    lib.amr_mlp_init.argtypes = [vp, vp, ctypes.c_uint64, vp]
    lib.amr_mlp_init.restype = i32
    lib.amr_mlp_grad.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]
    lib.amr_mlp_grad.restype = i32
    lib.amr_mlp_train_epoch.argtypes = [ctypes.POINTER(AmrMlpState), vp, vp, i64, i32,
                                        ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double), vp]
    lib.amr_mlp_train_epoch.restype = i32
    lib.amr_mlp_infer.argtypes = [vp, vp, i64, vp, vp]
    lib.amr_mlp_infer.restype = i32
    lib.amr_criterion_marks.argtypes = [vp, vp]
    lib.amr_criterion_marks.restype = i32
    lib.amr_propose_marks.argtypes = [vp, vp, ctypes.c_float, i32, vp]
    lib.amr_propose_marks.restype = i32
    lib.amr_mass_audit_noalloc.argtypes = [i32, i32, i32, i64, vp, vp, ctypes.c_uint32, vp, vp,
                                           vp, vp, vp, vp]
    lib.amr_mass_audit_noalloc.restype = i32
    pp = ctypes.POINTER(vp)
    lib.amr_validate_tables.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp, i64,
                                        ctypes.POINTER(i64), vp]
    lib.amr_validate_tables.restype = i32
    lib.amr_check_tables.argtypes = [vp, ctypes.POINTER(i64)]
    lib.amr_check_tables.restype = i32
    lib.amr_batch_arena_bytes.argtypes = [pp, i32]
    lib.amr_batch_arena_bytes.restype = sz
    lib.amr_batch_create.argtypes = [pp, i32, vp, sz, vp, pp]
    lib.amr_batch_create.restype = i32
    lib.amr_batch_refresh.argtypes = [vp]
    lib.amr_batch_refresh.restype = i32
    lib.amr_batch_step.argtypes = [vp, i32]
    lib.amr_batch_step.restype = i32
    cfgp = ctypes.POINTER(AmrBatchConfig)
    lib.amr_batch_configure.argtypes = [vp, cfgp]
    lib.amr_batch_configure.restype = i32
    lib.amr_batch_get_config.argtypes = [vp, cfgp]
    lib.amr_batch_get_config.restype = i32
    lib.amr_batch_autotune.argtypes = [vp, i32, i32, cfgp, ctypes.POINTER(ctypes.c_float)]
    lib.amr_batch_autotune.restype = i32
    lib.amr_batch_sync.argtypes = [vp]
    lib.amr_batch_sync.restype = i32
    lib.amr_batch_check_timeout.argtypes = [vp, ctypes.c_longlong]
    lib.amr_batch_check_timeout.restype = i32
    lib.amr_batch_plan.argtypes = [i32, i32, i32, vp, vp, vp, vp, i32, i32, ctypes.c_uint32, i32,
                                   vp, vp, vp, vp]
    lib.amr_batch_plan.restype = i32
    lib.amr_batch_launches.argtypes = [vp]
    lib.amr_batch_launches.restype = i64
    lib.amr_batch_free.argtypes = [vp]
    lib.amr_batch_free.restype = i32
    lib.amr_cells_table.argtypes = [i32, i32, i32, i32, i32, vp, vp]
    lib.amr_cells_table.restype = i32
    lib.amr_cells_step.argtypes = [i32, i32, i32, i32, i32, i32, ctypes.c_double, vp, vp, vp,
                                   i32, vp]
    lib.amr_cells_step.restype = i32
    lib.amr_cells_rest.argtypes = [i32, i32, i32, i32, i32, vp, vp]
    lib.amr_cells_rest.restype = i32
    _lib = lib
    return lib


class AmrError(RuntimeError):
    def __init__(self, code, where):
        lib = load_library()
        super().__init__("%s: %s (%s)" % (where, lib.amr_strerror(code).decode(),
                                          lib.amr_last_error().decode()))
        self.code = code


def make_config(cfg, storage="f32", use_graphs=True, kernel_variant=0):
    """Fill an AmrConfig from a workload dictionary (see workloads/)."""
    c = AmrConfig()
    c.dim, c.q = cfg["dim"], cfg["q"]
    c.storage = STORAGE[storage]
    c.nx, c.ny, c.nz = cfg["nx"], cfg["ny"], cfg["nz"]
    c.max_levels = cfg["max_levels"]
    c.crit_start, c.crit_inc = cfg["crit_start"], cfg["crit_inc"]
    c.max_blocks = cfg["max_blocks"]
    c.nu0 = cfg["nu0"]
    c.length_x = cfg.get("length_x", 1.0)
    if cfg.get("solid") is not None:
        c.has_solid = 1
        for i, v in enumerate(cfg["solid"]):
            c.solid[i] = v
    for i, face in enumerate(cfg["faces"]):
        c.faces[i].kind = FACE[face[0]]
        for a, v in enumerate(face[1]):
            c.faces[i].u[a] = v
        c.faces[i].rho_w = face[2] if len(face) > 2 else 1.0
    c.use_graphs = 1 if use_graphs else 0
    c.kernel_variant = int(kernel_variant)
    c.refine_dist = float(cfg.get("refine_dist", 0.0))
    c.refine_dist_targets = int(cfg.get("refine_dist_targets", 0))
    c.refine_dist_freeze = int(cfg.get("refine_dist_freeze", 0))
    ids = cfg.get("root_ids")
    if ids is not None:
        arr = np.ascontiguousarray(ids, dtype=np.int32)
        c._root_ids = arr                               # kept alive with the struct
        c.root_ids = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    c.interp = {"linear": 0, "cubic": 3}[cfg.get("interp", "linear")]
    c.check_tables = int(cfg.get("check_tables", 0))
    return c


class AmrLBM:
    """One block-forest AMR-LBM instance on the current CUDA device."""

    def __init__(self, cfg, storage="f32", stream=None, use_graphs=True, device=None,
                 kernel_variant=0):
        import torch
        self.lib = lib = load_library()
        self.cfg = cfg
        self.dim, self.q = cfg["dim"], cfg["q"]
        self.m = 4 ** self.dim
        self.nk = 3 ** self.dim
        self.cap = cfg["max_blocks"]
        self.lmax = cfg["max_levels"]
        self.storage = storage
        self.c = make_config(cfg, storage, use_graphs, kernel_variant)
        nbytes = lib.amr_arena_bytes(ctypes.byref(self.c))
        if nbytes == 0:
            raise AmrError(AMR_E_INVAL, "amr_arena_bytes")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.arena.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.h = ctypes.c_void_p()
        rc = lib.amr_init(ctypes.byref(self.c), ctypes.c_void_p(base + off), nbytes,
                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_init")

    # ------------------------------------------------------------ calls
    def _check(self, rc, where, ok=(AMR_OK,)):
        if rc not in ok:
            raise AmrError(rc, where)
        return rc

    def step(self, n=1):
        self._check(self.lib.amr_step(self.h, int(n)), "amr_step")

    def adapt(self, marks=None):
        """Adapt the mesh; marks: optional int8 torch CUDA tensor (+1/-1/0) of
        length max_blocks.  Returns (status code, stats dict)."""
        st = AmrAdaptStats()
        ptr = None
        if marks is not None:
            assert marks.dtype.itemsize == 1 and marks.numel() >= self.cap and marks.is_cuda
            ptr = ctypes.c_void_p(marks.data_ptr())
        rc = self.lib.amr_adapt(self.h, ptr, ctypes.byref(st))
        self._check(rc, "amr_adapt", ok=(AMR_OK, AMR_E_CAPACITY))
        return rc, {k: getattr(st, k) for k, _ in AmrAdaptStats._fields_ if k != "pad_"}

    def field_bytes(self, what):
        n = self.lib.amr_fields(self.h, what, None, 0, 0)
        if n < 0:
            raise AmrError(int(n), "amr_fields")
        return int(n)

    # mesh tables above this size are exported to device memory and copied
    # from there (the library stages host exports of tables through 32 MiB)
    TABLE_STAGING_BYTES = 32 << 20

    def fields_host(self, what, dtype):
        n = self.field_bytes(what)
        if n > self.TABLE_STAGING_BYTES and what not in (AMR_F, AMR_RHO_U, AMR_FEATURES):
            import torch
            tdt = {np.dtype(np.int32): torch.int32, np.dtype(np.float64): torch.float64,
                   np.dtype(np.uint8): torch.uint8, np.dtype(np.int64): torch.int64}[np.dtype(dtype)]
            return self.fields_device(what, tdt).cpu().numpy()
        out = np.empty(n // np.dtype(dtype).itemsize, dtype=dtype)
        rc = self.lib.amr_fields(self.h, what, out.ctypes.data_as(ctypes.c_void_p), n, 0)
        if rc < 0:
            raise AmrError(int(rc), "amr_fields")
        return out

    def fields_device(self, what, torch_dtype):
        import torch
        n = self.field_bytes(what)
        out = torch.empty(n // torch.empty(0, dtype=torch_dtype).element_size(),
                          dtype=torch_dtype, device=self.device)
        rc = self.lib.amr_fields(self.h, what, ctypes.c_void_p(out.data_ptr()), n, 1)
        if rc < 0:
            raise AmrError(int(rc), "amr_fields")
        return out

    # ------------------------------------------------------ conveniences
    def populations(self):
        """f [cap, M, Q] (float64) at each block's current time."""
        f = self.fields_host(AMR_F, np.float64).reshape(self.q, self.cap, self.m)
        return np.ascontiguousarray(f.transpose(1, 2, 0))

    def set_populations(self, f):
        """Overwrite the populations from f [cap, M, Q] (float64)."""
        arr = np.ascontiguousarray(np.asarray(f, np.float64).transpose(2, 0, 1))
        self._check(self.lib.amr_set_fields(self.h, AMR_F, arr.ctypes.data_as(ctypes.c_void_p),
                                            arr.nbytes, 0), "amr_set_fields")

    def rho_u(self):
        a = self.fields_host(AMR_RHO_U, np.float64).reshape(self.cap, self.m, 1 + self.dim)
        return a[..., 0], a[..., 1:]

    def blocks(self):
        b = self.fields_host(AMR_BLOCKS, np.int32).reshape(4, self.cap)
        return dict(level=b[0], status=b[1], child0=b[2], parent=b[3])

    def coords(self):
        return self.fields_host(AMR_COORDS, np.float64).reshape(self.cap, self.dim)

    def nbr(self):
        return self.fields_host(AMR_NBR, np.int32).reshape(self.cap, self.nk)

    def nbr_child(self):
        return self.fields_host(AMR_NBR_CHILD, np.int32).reshape(self.cap, self.nk)

    def masks(self):
        return self.fields_host(AMR_MASKS, np.uint8).reshape(self.cap, self.m)

    def counts(self):
        c = self.fields_host(AMR_COUNTS, np.int64)
        lmax = int(c[0])
        per = c[4:4 + 4 * lmax].reshape(lmax, 4)
        return dict(n_gaps=int(c[1]), coarse_steps=int(c[2]), launches=int(c[3]),
                    n_ids=per[:, 0].tolist(),
                    n_active=per[:, 1].tolist(), n_leaves=per[:, 2].tolist(),
                    n_parents=per[:, 3].tolist())

    def id_sets(self):
        ids = self.fields_host(AMR_IDSETS, np.int32).reshape(self.lmax, self.cap)
        n = self.counts()["n_ids"]
        return [ids[L, :n[L]].tolist() for L in range(self.lmax)]

    def gaps(self):
        g = self.fields_host(AMR_GAPS, np.int32)
        return g[:self.counts()["n_gaps"]].tolist()

    def mass(self):
        return self.fields_host(AMR_MASS, np.float64)

    def force(self):
        return self.fields_host(AMR_FORCE, np.float64)

    def profile(self, mode=1):
        """0 off, 1 events around every launch (no graphs), 2 events inside the
        coarse-step graphs (one sample per profile_read)."""
        self._check(self.lib.amr_profile(self.h, int(mode)), "amr_profile")

    def profile_read(self, reset=True):
        arr = (AmrKernelProfile * 16)()
        n = self.lib.amr_profile_read(self.h, arr, 16, 1 if reset else 0)
        if n < 0:
            raise AmrError(n, "amr_profile_read")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms,
                                           bytes=arr[i].bytes, cells=arr[i].cells)
                for i in range(n)}

    def launches(self):
        return self.counts()["launches"]

    def features(self):
        """Block summaries [cap, 27] (float32, device tensor; runs a sync)."""
        import torch
        return self.fields_device(AMR_FEATURES, torch.float32).reshape(self.cap, MLP_INPUTS)

    def criterion_marks(self):
        """Marks of the plain criterion without adapting (int8 device tensor)."""
        import torch
        out = torch.zeros(self.cap, dtype=torch.int8, device=self.device)
        self._check(self.lib.amr_criterion_marks(self.h, ctypes.c_void_p(out.data_ptr())),
                    "amr_criterion_marks")
        return out

    def propose_marks(self, params_half, threshold=0.5, with_criterion=True):
        """Marks from the learned proposal (merged with the plain criterion)."""
        import torch
        out = torch.zeros(self.cap, dtype=torch.int8, device=self.device)
        self._check(self.lib.amr_propose_marks(self.h, ctypes.c_void_p(params_half.data_ptr()),
                                               float(threshold), 1 if with_criterion else 0,
                                               ctypes.c_void_p(out.data_ptr())),
                    "amr_propose_marks")
        return out

    def updates_per_coarse_step(self):
        """Leaf-cell updates of one coarse step (Section 5.1 definition)."""
        c = self.counts()
        return sum((2 ** L) * c["n_leaves"][L] * self.m for L in range(self.lmax))

    def check_tables(self):
        """(bad entries, first bad block or -1, AMR_CHECK_* code) of the
        device validation of the block tables, lists and averaging groups."""
        out = (ctypes.c_int64 * 3)()
        rc = self.lib.amr_check_tables(self.h, out)
        self._check(rc, "amr_check_tables", ok=(AMR_OK, AMR_E_INVAL))
        return tuple(int(v) for v in out)

    def checkpoint(self):
        """Host image (numpy uint8) of the whole instance state."""
        n = self.lib.amr_checkpoint_bytes(self.h)
        if n < 0:
            raise AmrError(n, "amr_checkpoint_bytes")
        buf = np.empty(n, np.uint8)
        self._check(self.lib.amr_checkpoint(self.h, buf.ctypes.data_as(ctypes.c_void_p), n),
                    "amr_checkpoint")
        return buf

    def restore(self, image):
        """Load a checkpoint image made by an instance of the same configuration."""
        buf = np.ascontiguousarray(image, np.uint8)
        self._check(self.lib.amr_restore(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes),
                    "amr_restore")

    def close(self):
        if self.h:
            self.lib.amr_free(self.h)
            self.h = ctypes.c_void_p()
        self.arena = None             # the device arena goes back to torch's allocator

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


AMR_BATCH_GRAPH, AMR_BATCH_PERSISTENT, AMR_BATCH_MEMBERS = 0, 1, 2
BATCH_FORMS = {"graph": AMR_BATCH_GRAPH, "persistent": AMR_BATCH_PERSISTENT,
               "members": AMR_BATCH_MEMBERS}
# candidate order of amr_batch_autotune's ms_out
BATCH_CANDIDATES = ([("graph", t, t // 64) for t in (512, 256, 128, 64)] +
                    [("persistent", t, m) for m in (1, 2, 4, 8) for t in (64, 128, 256)] +
                    [("members", 0, 0)])


class AmrBatchConfig(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("tile_blocks", ctypes.c_int32), ("ctas", ctypes.c_int32)]

    def as_dict(self):
        form = {v: k for k, v in BATCH_FORMS.items()}[self.mode]
        return {"form": form, "threads": self.threads, "tile_blocks": self.tile_blocks,
                "ctas": self.ctas}


class AmrBatch:
    """Batch of AmrLBM instances (same velocity set and storage) advanced
    together, in the graph form or the persistent form (amr_batch_configure)."""

    def __init__(self, members, stream=None):
        import torch
        self.lib = lib = load_library()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        self._arr = arr
        n = len(self.members)
        nbytes = lib.amr_batch_arena_bytes(arr, n)
        if nbytes == 0:
            raise AmrError(AMR_E_INVAL, "amr_batch_arena_bytes")
        dev = self.members[0].device
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.arena.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.h = ctypes.c_void_p()
        rc = lib.amr_batch_create(arr, n, ctypes.c_void_p(base + off), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_create")

    def refresh(self):
        rc = self.lib.amr_batch_refresh(self.h)
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_refresh")

    def step(self, n=1):
        rc = self.lib.amr_batch_step(self.h, int(n))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_step")

    def configure(self, form="graph", threads=512, tile_blocks=0, ctas=0):
        cfg = AmrBatchConfig(BATCH_FORMS[form], int(threads), int(tile_blocks), int(ctas))
        rc = self.lib.amr_batch_configure(self.h, ctypes.byref(cfg))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_configure")

    def config(self):
        cfg = AmrBatchConfig()
        rc = self.lib.amr_batch_get_config(self.h, ctypes.byref(cfg))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_get_config")
        return cfg.as_dict()

    def autotune(self, trial_steps=2, forms=("graph", "persistent", "members")):
        """Times every candidate; returns (chosen config, {candidate: ms per
        coarse step}).  The members advance."""
        bits = sum(1 << BATCH_FORMS[f] for f in forms)
        cfg = AmrBatchConfig()
        ms = (ctypes.c_float * len(BATCH_CANDIDATES))()
        rc = self.lib.amr_batch_autotune(self.h, int(trial_steps), bits, ctypes.byref(cfg), ms)
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_autotune")
        times = {c: float(v) for c, v in zip(BATCH_CANDIDATES, ms) if v >= 0}
        return cfg.as_dict(), times

    def sync(self):
        rc = self.lib.amr_batch_sync(self.h)
        if rc != AMR_OK:
            raise AmrError(rc, "amr_batch_sync")

    def check_timeout(self, limit_cycles):
        """Return code of amr_batch_check_timeout (AMR_E_TIMEOUT expected)."""
        return int(self.lib.amr_batch_check_timeout(self.h, int(limit_cycles)))

    def launches(self):
        return int(self.lib.amr_batch_launches(self.h))

    def close(self):
        if self.h:
            self.lib.amr_batch_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Per-block MLP of the learned refinement proposal (device tensors)."""

    def __init__(self, device, seed=0, stream=None):
        import torch
        self.lib = lib = load_library()
        self.n = lib.amr_mlp_param_count()
        f32 = dict(dtype=torch.float32, device=device)
        self.params = torch.empty(self.n, **f32)
        self.half = torch.empty(self.n, dtype=torch.float16, device=device)
        self.m = torch.zeros(self.n, **f32)
        self.v = torch.zeros(self.n, **f32)
        self.grad = torch.zeros(self.n, **f32)
        self.loss = torch.zeros(1, **f32)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.state = AmrMlpState(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                 self.half.data_ptr(), self.grad.data_ptr(),
                                 self.loss.data_ptr(), 0)
        rc = lib.amr_mlp_init(ctypes.c_void_p(self.params.data_ptr()),
                              ctypes.c_void_p(self.half.data_ptr()), int(seed),
                              ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_mlp_init")

    def train_epoch(self, x, y, batch=1024, lr=1e-3, pos_weight=1.0, seed=0):
        out = ctypes.c_double(0.0)
        rc = self.lib.amr_mlp_train_epoch(ctypes.byref(self.state), ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), int(x.shape[0]),
                                          int(batch), float(lr), float(pos_weight), int(seed),
                                          ctypes.byref(out),
                                          ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_mlp_train_epoch")
        return out.value

    def grad_of(self, x, y, pos_weight=1.0):
        rc = self.lib.amr_mlp_grad(ctypes.c_void_p(self.params.data_ptr()),
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                   int(x.shape[0]), float(pos_weight),
                                   ctypes.c_void_p(self.grad.data_ptr()),
                                   ctypes.c_void_p(self.loss.data_ptr()),
                                   ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_mlp_grad")
        return self.grad, self.loss

    def infer(self, x):
        import torch
        prob = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        rc = self.lib.amr_mlp_infer(ctypes.c_void_p(self.half.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                    ctypes.c_void_p(prob.data_ptr()),
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_mlp_infer")
        return prob


def cells_table(dim, q, shape, id_of_pos=None):
    """Neighbour table int32 [q][n] of the cell-based solver, filled by the
    library on the host: entry [p][id of position i] is the ID of the
    position one link c_p downstream of i (periodic).  id_of_pos: element ID
    of each x-fastest position (None: the positions themselves)."""
    lib = load_library()
    shape = list(shape) + [1] * (3 - len(shape))
    n = int(np.prod(shape))
    table = np.empty(q * n, np.int32)
    ids = None
    if id_of_pos is not None:
        ids = np.ascontiguousarray(id_of_pos, dtype=np.int32)
        if ids.size != n:
            raise AmrError(AMR_E_INVAL, "cells_table: id_of_pos has %d entries, not %d" % (ids.size, n))
    rc = lib.amr_cells_table(dim, q, shape[0], shape[1], shape[2],
                             None if ids is None else ids.ctypes.data_as(ctypes.c_void_p),
                             table.ctypes.data_as(ctypes.c_void_p))
    if rc != AMR_OK:
        raise AmrError(rc, "amr_cells_table")
    return table.reshape(q, n)


class Cells:
    """Cell-based uniform periodic solver (the cell arrangement of the
    comparison of cell- and block-based grids): FP32 populations [q][n] by
    element ID in two device buffers, and for the retrieved connectivity the
    neighbour table on the device.  id_of_pos None selects the computed
    connectivity with x-fastest IDs; otherwise neighbours are read from the
    table built for those IDs."""

    def __init__(self, dim, q, shape, nu0, id_of_pos=None, stream=None, device=None):
        import torch
        self.lib = load_library()
        self.dim, self.q = dim, q
        self.shape = list(shape)
        self.dims = self.shape + [1] * (3 - len(self.shape))
        self.n = int(np.prod(self.shape))
        self.nu0 = float(nu0)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ids = None if id_of_pos is None else np.ascontiguousarray(id_of_pos, dtype=np.int32)
        self.connectivity = AMR_CELLS_CALCULATED if self.ids is None else AMR_CELLS_RETRIEVED
        self.table = None
        if self.ids is not None:
            self.table = torch.from_numpy(cells_table(dim, q, self.shape, self.ids)).to(dev)
        self.buf = [torch.empty(q * self.n, dtype=torch.float32, device=dev) for _ in range(2)]
        self.cur = 0

    def set_rest(self):
        """Rest equilibrium (rho = 1, u = 0) in every cell."""
        rc = self.lib.amr_cells_rest(self.dim, self.q, self.dims[0], self.dims[1], self.dims[2],
                                     ctypes.c_void_p(self.buf[self.cur].data_ptr()),
                                     ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_cells_rest")

    def set_f(self, f_pos):
        """Load populations given per x-fastest position, array [n, q]."""
        import torch
        f_pos = np.asarray(f_pos, np.float32).reshape(self.n, self.q)
        f_id = np.empty((self.q, self.n), np.float32)
        if self.ids is None:
            f_id[:] = f_pos.T
        else:
            f_id[:, self.ids] = f_pos.T
        self.buf[self.cur].copy_(torch.from_numpy(f_id.reshape(-1)))

    def f(self):
        """Populations per x-fastest position, array [n, q] (synchronises)."""
        f_id = self.buf[self.cur].cpu().numpy().reshape(self.q, self.n)
        return (f_id if self.ids is None else f_id[:, self.ids]).T.copy()

    def step(self, n=1):
        a, b = self.buf[self.cur], self.buf[1 - self.cur]
        rc = self.lib.amr_cells_step(
            self.dim, self.q, self.dims[0], self.dims[1], self.dims[2], self.connectivity,
            self.nu0, None if self.table is None else ctypes.c_void_p(self.table.data_ptr()),
            ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), int(n),
            ctypes.c_void_p(self.stream.cuda_stream))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_cells_step")
        self.cur ^= int(n) & 1

"""GPU parity tests: the CUDA library (through its C ABI) against the CPU oracle
on the same seeded inputs.

Bars: integer results (block tables, neighbour tables, ID sets, gap stack,
cell classes) bit-exact; fields relative L2 <= 1e-12 in FP64 and <= 1e-5 in
FP32 (the FP32 bar also covers the rounding of the FP64 initial state)."""
import ctypes

import numpy as np
import pytest

import workloads as W
from cellwise import assert_cells, oracle_classes
from oracle.forest import Forest
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def new_gpu(cfg, storage, variant=0):
    from paper_2308_08085_gb300 import AmrLBM
    return AmrLBM(cfg, storage=storage, kernel_variant=variant)


def randomize(ref, seed, noise=1e-3):
    """Seeded random state (equilibrium of random rho, u plus noise) on every
    active block of the oracle; solid cells keep the rest state."""
    ids = np.array(ref.mesh.active_ids())
    n = len(ids) * ref.m
    rho, u = W.random_macro(seed, n, ref.dim)
    f = equilibrium(ref.vs, rho, u) + W.random_noise(seed + 1, (n, ref.vs.q), noise)
    f = f.reshape(len(ids), ref.m, ref.vs.q)
    sol = ref.solid[ids]
    f[sol] = ref.rest
    ref.f[ids] = f


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_fields(got, ref, ids, storage, what=""):
    """Relative L2 over all compared cells within TOL, and the worst cell of
    each class (ghost, interface, interior) within the per-cell bar."""
    want = ref.f[ids]
    err = rel_l2(got, want)
    assert err <= TOL[storage], (what, storage, err)
    assert_cells(got, want, oracle_classes(ref.mesh, ids), ref.vs.w, storage, what=what)


def marks_tensor(m):
    return torch.from_numpy(np.ascontiguousarray(m, dtype=np.int8)).cuda()


# ------------------------------------------------------------ single level
SINGLE = [
    ("cavity2d", lambda: W.cavity(dim=2, q=9, n=20, ny=12, max_levels=1), ("f64", "f32")),
    ("cavity3d_q19", lambda: W.cavity(dim=3, q=19, n=12, ny=8, nz=16, max_levels=1), ("f64", "f32")),
    ("periodic3d_q27", lambda: W.periodic_box(dim=3, q=27, n=8, ny=12, nz=4), ("f64", "f32")),
    ("cylinder_q19", lambda: W.channel_cylinder(q=19, nx=24, ny=16, nz=8, side=4, cx=8, cy=8,
                                               max_levels=1), ("f64", "f32")),
    ("cylinder_q27", lambda: W.channel_cylinder(q=27, nx=16, ny=12, nz=4, side=4, cx=6, cy=6,
                                               max_levels=1), ("f64",)),
]


@pytest.mark.parametrize("variant", list(range(0, 6)))
@pytest.mark.parametrize("name,mk,storages", SINGLE, ids=[c[0] for c in SINGLE])
def test_single_level_collide_stream(name, mk, storages, variant):
    """Every collide-stream kernel variant (fused BGK + pull streaming): 512 /
    256 / 128 / 64 threads per CTA (1 to 4), 128 threads with the tighter
    register budget (5) and the default (0), on walls, moving lids, periodic
    boxes, solid prisms and the outlet."""
    for storage in storages:
        cfg = mk()
        ref = ForestLBM(cfg)
        randomize(ref, 21)
        gpu = new_gpu(cfg, storage, variant)
        gpu.set_populations(ref.f)
        for _ in range(5):
            ref.step(1)
            gpu.step(1)
        ids = ref.mesh.active_ids()
        check_fields(gpu.populations()[ids], ref, ids, storage, name)
        gpu.close()


# ----------------------------------------------------------- mesh tables
def with_roots(cfg, ids):
    cfg = dict(cfg)
    cfg["root_ids"] = ids(cfg)
    return cfg


MESHES = [
    ("2d_cavity_3x3", lambda: W.cavity(dim=2, n=12, max_levels=4, max_blocks=9 * 40)),
    ("2d_periodic_2x3", lambda: W.periodic_box(dim=2, n=8, ny=12, max_levels=3, max_blocks=200)),
    ("3d_cavity_2x2x2", lambda: W.cavity(dim=3, n=8, max_levels=3, max_blocks=8 * 30)),
    ("3d_periodic_3x2x2", lambda: W.periodic_box(dim=3, n=12, ny=8, nz=8, max_levels=3,
                                                 max_blocks=12 * 25)),
    ("2d_cavity_4x3_shuffled", lambda: with_roots(
        W.cavity(dim=2, n=16, ny=12, max_levels=3, max_blocks=12 * 20),
        lambda c: W.shuffled_root_ids(c, 5))),
    ("3d_periodic_3x2x2_morton", lambda: with_roots(
        W.periodic_box(dim=3, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 25),
        W.morton_root_ids)),
]


def same(name, got, want):
    got, want = np.asarray(got), np.asarray(want)
    if got.shape == want.shape and np.array_equal(got, want):
        return
    rows = np.nonzero(np.any((got != want).reshape(len(got), -1), axis=1))[0][:5]
    msg = "; ".join("row %d: got %s want %s" % (r, got[r].tolist(), want[r].tolist())
                    for r in rows)
    raise AssertionError("%s differs: %s" % (name, msg))


def compare_tables(gpu, mesh: Forest):
    blk = gpu.blocks()
    for k in ("level", "status", "child0", "parent"):
        same(k, blk[k], getattr(mesh, k))
    same("nbr", gpu.nbr(), mesh.nbr)
    ncg = gpu.nbr_child()
    act = mesh.active_ids()
    for b in act:
        assert np.array_equal(ncg[b], mesh.nbr_child(b)), b
    assert gpu.id_sets() == mesh.id_sets
    assert gpu.gaps() == mesh.gap
    assert np.array_equal(gpu.coords()[act], mesh.X[act])
    masks = gpu.masks()
    for b in act:
        assert np.array_equal(masks[b], mesh.cell_classes(b)), b
    cnt = gpu.counts()
    assert cnt["n_gaps"] == len(mesh.gap)
    for L in range(mesh.lmax):
        assert cnt["n_active"][L] == len(mesh.active_list(L))
        assert cnt["n_parents"][L] == len(mesh.parent_list(L))
        assert cnt["n_leaves"][L] == sum(1 for b in mesh.id_sets[L] if mesh.status[b] == 1)


@pytest.mark.parametrize("name,mk", MESHES, ids=[m[0] for m in MESHES])
def test_mesh_tables_bit_exact(name, mk):
    cfg = mk()
    mesh = Forest(cfg)
    gpu = new_gpu(cfg, "f64" if cfg["dim"] == 2 else "f32")
    compare_tables(gpu, mesh)
    for it in range(10):
        m = W.random_marks(300 + it, cfg["max_blocks"], 0.35, 0.3)
        res = mesh.adapt(m)
        rc, st = gpu.adapt(marks_tensor(m))
        assert st["n_refined"] == res["n_refined"]
        assert st["n_coarsened"] == res["n_coarsened"]
        assert bool(st["capacity_error"]) == res["capacity_error"]
        compare_tables(gpu, mesh)
    gpu.close()


def test_capacity_error_keeps_coarsening():
    cfg = W.cavity(dim=2, n=8, max_levels=3, max_blocks=4 + 8)
    mesh = Forest(cfg)
    gpu = new_gpu(cfg, "f64")
    m = np.zeros(cfg["max_blocks"], np.int8)
    m[[0, 1]] = 1
    mesh.adapt(m)
    gpu.adapt(marks_tensor(m))
    m[:] = 0
    m[[0]] = -1          # coarsen 0 and try to refine 2 and 3 (no room)
    m[[2, 3]] = 1
    res = mesh.adapt(m)
    rc, st = gpu.adapt(marks_tensor(m))
    assert res["capacity_error"] and st["capacity_error"] == 1
    from paper_2308_08085_gb300.amr import AMR_E_CAPACITY
    assert rc == AMR_E_CAPACITY
    assert st["n_coarsened"] == 1
    compare_tables(gpu, mesh)
    gpu.close()


# ------------------------------------------------------ multi-level steps
def static_mesh(cfg, seq):
    ref = ForestLBM(cfg)
    gpu = new_gpu(cfg, "f64")
    for ids in seq:
        m = np.zeros(cfg["max_blocks"], np.int8)
        m[ids(ref.mesh)] = 1
        ref.adapt(m)
        gpu.adapt(marks_tensor(m))
    return ref, gpu


def leaves_where(pred):
    return lambda mesh: [b for b in mesh.active_ids() if mesh.status[b] == 1 and pred(mesh, b)]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_three_level_step_2d(storage):
    cfg = W.cavity(dim=2, q=9, n=24, ny=16, max_levels=3, max_blocks=24 * 30)
    near_lid = leaves_where(lambda m, b: m.X[b][1] >= 8 and 4 <= m.X[b][0] < 20)
    ref, gpu64 = static_mesh(cfg, [near_lid, near_lid])
    gpu64.close()
    gpu = new_gpu(cfg, storage)
    # replay the same marks on the GPU instance of the requested storage
    ref2 = ForestLBM(cfg)
    for _ in range(2):
        m = np.zeros(cfg["max_blocks"], np.int8)
        m[near_lid(ref2.mesh)] = 1
        ref2.adapt(m)
        gpu.adapt(marks_tensor(m))
    assert ref2.mesh.counts()[2] > 0
    randomize(ref2, 5)
    gpu.set_populations(ref2.f)
    ref2.step(3)
    gpu.step(3)
    ref2.sync()
    gpu.rho_u()                      # runs the level synchronisation
    ids = ref2.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref2, ids, storage)
    gpu.close()


@pytest.mark.parametrize("q,storage,variant", [(19, "f64", 1), (19, "f32", 1), (27, "f64", 1),
                                               (19, "f32", 2), (27, "f32", 3), (19, "f32", 4),
                                               (19, "f64", 5), (27, "f32", 0), (19, "f32", 0)])
def test_two_level_step_3d(q, storage, variant):
    cfg = W.cavity(dim=3, q=q, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 40)
    two_level_case(cfg, storage, variant)


def two_level_case(cfg, storage, variant=0):
    sel = leaves_where(lambda m, b: m.X[b][2] >= 4 and m.X[b][0] >= 4)
    ref = ForestLBM(cfg)
    gpu = new_gpu(cfg, storage, variant)
    for _ in range(2):
        m = np.zeros(cfg["max_blocks"], np.int8)
        m[sel(ref.mesh)] = 1
        ref.adapt(m)
        gpu.adapt(marks_tensor(m))
    assert ref.mesh.counts()[2] > 0
    randomize(ref, 9)
    gpu.set_populations(ref.f)
    ref.step(2)
    gpu.step(2)
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, storage)
    gpu.close()


# ------------------------------------------- end to end with the criterion
def run_pair(cfg, storage, steps, every):
    ref = ForestLBM(cfg)
    gpu = new_gpu(cfg, storage)
    for t in range(steps // every):
        ref.step(every)
        gpu.step(every)
        ref.adapt()
        gpu.adapt()
    return ref, gpu


def test_cavity2d_criterion_end_to_end_f64():
    cfg = W.cavity(dim=2, q=9, n=32, re=100.0, max_levels=3, max_blocks=64 * 24)
    ref, gpu = run_pair(cfg, "f64", 200, 50)
    compare_tables(gpu, ref.mesh)
    assert sum(ref.mesh.counts()[1:]) > 0          # the criterion refined something
    ref.step(10)
    gpu.step(10)
    ref.sync()
    rho_g, u_g = gpu.rho_u()
    ids = ref.mesh.active_ids()
    rho_r, u_r = ref.macroscopic()
    assert rel_l2(u_g[ids], u_r[ids]) <= 1e-12
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    gpu.close()


def test_cavity3d_criterion_end_to_end_f64():
    cfg = W.cavity(dim=3, q=19, n=16, re=100.0, max_levels=3, max_blocks=64 * 20)
    ref, gpu = run_pair(cfg, "f64", 60, 20)
    compare_tables(gpu, ref.mesh)
    assert sum(ref.mesh.counts()[1:]) > 0
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    gpu.close()


def test_shuffled_roots_criterion_end_to_end_f64():
    """Root blocks numbered by a seeded permutation (block IDs no longer follow
    space): tables bit-exact and fields within 1e-12 through criterion-driven
    adaptation."""
    cfg = with_roots(W.cavity(dim=3, q=19, n=16, re=100.0, max_levels=3, max_blocks=64 * 20),
                     lambda c: W.shuffled_root_ids(c, 17))
    ref, gpu = run_pair(cfg, "f64", 60, 20)
    compare_tables(gpu, ref.mesh)
    assert sum(ref.mesh.counts()[1:]) > 0
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    gpu.close()


def test_mass_audit_matches_oracle():
    cfg = W.cavity(dim=2, q=9, n=16, max_levels=2, max_blocks=16 * 6)
    ref = ForestLBM(cfg)
    gpu = new_gpu(cfg, "f64")
    m = np.zeros(cfg["max_blocks"], np.int8)
    m[[5, 6, 9, 10]] = 1
    ref.adapt(m)
    gpu.adapt(marks_tensor(m))
    randomize(ref, 3)
    gpu.set_populations(ref.f)
    ms = gpu.mass()
    rho, u = ref.macroscopic()
    mass = mom_x = 0.0
    for b in ref.mesh.active_ids():
        if ref.mesh.status[b] != 1:
            continue
        vol = 0.25 ** ref.mesh.level[b]
        mass += rho[b].sum() * vol
        mom_x += (rho[b] * u[b][:, 0]).sum() * vol
    assert abs(ms[0] - mass) <= 1e-12 * mass
    assert abs(ms[1] - mom_x) <= 1e-12 * max(1.0, abs(mom_x))
    gpu.close()


# ------------------------------------------------ cylinder, distance rule, force
def test_cavity_wall_distance_rule_end_to_end():
    """Distance refinement towards the walls with freezing (REFINED_PERMANENT),
    together with the vorticity criterion: tables bit-exact, fields 1e-12."""
    cfg = W.cavity(dim=3, q=19, n=16, re=200.0, max_levels=3, max_blocks=64 * 40,
                   refine_dist=0.1, refine_dist_freeze=1)
    ref, gpu = run_pair(cfg, "f64", 60, 20)
    compare_tables(gpu, ref.mesh)
    assert np.any(ref.mesh.status == 4)
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    gpu.close()


@pytest.mark.parametrize("span_periodic", [False, True])
def test_cylinder_distance_rule_force_end_to_end(span_periodic):
    """Prism, outlet, distance refinement with freezing and the drag; with a
    periodic one-block span (the quasi-2D case) as well."""
    cfg = W.channel_cylinder(q=19, nx=48, ny=24, nz=4 if span_periodic else 8, side=4, cx=16,
                             cy=13 if span_periodic else 12, max_levels=3,
                             max_blocks=72 * (80 if span_periodic else 30), refine_dist=0.15,
                             span_periodic=span_periodic)
    ref, gpu = run_pair(cfg, "f64", 60, 20)
    compare_tables(gpu, ref.mesh)
    assert np.any(ref.mesh.status == 4)             # frozen blocks around prism and outlet
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    f_ref = ref.mea_force()
    f_gpu = gpu.force()
    assert abs(f_ref[0]) > 0
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    gpu.close()


def test_cylinder_2d_distance_rule_force_end_to_end():
    """The paper's 2D flow past a square cylinder (Section 5.3) in small: D2Q9
    with a solid square, inlet and far field by moving-wall bounce-back, the
    anti-bounce-back outlet, distance refinement with freezing and the
    vorticity criterion; tables bit-exact, fields within 1e-12, the
    momentum-exchange force within 1e-11 of the oracle."""
    cfg = W.channel_cylinder(dim=2, nx=96, ny=48, side=4, cx=24, cy=25, max_levels=3,
                             max_blocks=288 * 40, refine_dist=0.05, crit_start=-1)
    ref, gpu = run_pair(cfg, "f64", 80, 20)
    assert ref.mesh.counts()[2] > 0
    compare_tables(gpu, ref.mesh)
    assert np.any(ref.mesh.status == 4)
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    f_ref, f_gpu = ref.mea_force(), gpu.force()
    assert len(f_ref) == 2 and abs(f_ref[0]) > 0 and f_gpu[2] == 0.0
    assert np.max(np.abs(f_gpu[:2] - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    gpu.close()


# ------------------------------------------------- cubic interpolation
def cubic(cfg):
    cfg = dict(cfg)
    cfg["interp"] = "cubic"
    return cfg


@pytest.mark.parametrize("q,storage", [(19, "f64"), (19, "f32"), (27, "f64")])
def test_cubic_two_level_step_3d(q, storage):
    """Cubic coarse-to-fine interpolation (Section 3.4.2): ghost cells of the
    normal step, every cell of new children, and the pre-adapt sync."""
    cfg = cubic(W.cavity(dim=3, q=q, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 40))
    two_level_case(cfg, storage)


def test_cubic_criterion_end_to_end_2d_f64():
    cfg = cubic(W.cavity(dim=2, q=9, n=32, re=100.0, max_levels=3, max_blocks=64 * 24))
    ref, gpu = run_pair(cfg, "f64", 200, 50)
    compare_tables(gpu, ref.mesh)
    assert sum(ref.mesh.counts()[1:]) > 0
    ref.step(10)
    gpu.step(10)
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    gpu.close()


def test_cubic_cylinder_end_to_end_f64():
    """Cubic interpolation next to the solid prism (solid cells are skipped)."""
    cfg = cubic(W.channel_cylinder(q=19, nx=48, ny=24, nz=8, side=4, cx=16, cy=12, max_levels=3,
                                   max_blocks=72 * 30, refine_dist=0.15))
    ref, gpu = run_pair(cfg, "f64", 40, 20)
    compare_tables(gpu, ref.mesh)
    ref.sync()
    gpu.rho_u()
    ids = ref.mesh.active_ids()
    check_fields(gpu.populations()[ids], ref, ids, "f64")
    f_ref, f_gpu = ref.mea_force(), gpu.force()
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    gpu.close()


# ------------------------------------------------------- 16-bit storage
@pytest.mark.parametrize("storage,unit_roundoff", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)])
def test_shifted_16bit_storage_within_rounding_bound(storage, unit_roundoff):
    """Populations stored as g = f - w_p in BF16 / FP16 (FP32 arithmetic).
    Every store rounds g to nearest with relative error <= u (unit roundoff);
    the error after n coarse steps of a two-level forest is bounded by the
    number of stores a value goes through, K = 1 + n * 2^(L_max-1) * 2
    (collide-stream plus interpolation/averaging), times u |g| / |f|."""
    cfg = W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=2, max_blocks=12 * 12)
    sel = leaves_where(lambda m, b: m.X[b][0] >= 4)
    ref = ForestLBM(cfg)
    gpu = new_gpu(cfg, storage)
    gpu32 = new_gpu(cfg, "f32")
    m = np.zeros(cfg["max_blocks"], np.int8)
    m[sel(ref.mesh)] = 1
    ref.adapt(m)
    gpu.adapt(marks_tensor(m))
    gpu32.adapt(marks_tensor(m))
    randomize(ref, 31)
    ids = ref.mesh.active_ids()
    g = ref.f[ids] - ref.vs.w
    ratio = np.linalg.norm(g) / np.linalg.norm(ref.f[ids])
    gpu.set_populations(ref.f)
    gpu32.set_populations(ref.f)
    n = 4
    ref.step(n)
    gpu.step(n)
    gpu32.step(n)
    ref.sync()
    gpu.rho_u()
    gpu32.rho_u()
    err = rel_l2(gpu.populations()[ids], ref.f[ids])
    err32 = rel_l2(gpu32.populations()[ids], ref.f[ids])
    K = 1 + n * 2 ** (cfg["max_levels"] - 1) * 2
    bound = K * unit_roundoff * ratio
    assert 0 < err <= bound, (err, bound)
    assert err32 < err / 10
    gpu.close()
    gpu32.close()


# ---------------------------------------------------- checkpoint / resume
def test_checkpoint_restore_resumes_bit_exactly():
    """A checkpoint image restored into a fresh instance (graphs off: the same
    kernels launched one by one) continues exactly as the original: tables and
    populations bit-identical after more steps and an adaptation."""
    cfg = W.cavity(dim=3, q=19, n=16, re=400.0, max_levels=3, max_blocks=64 * 20)
    a = new_gpu(cfg, "f32")
    for _ in range(2):
        a.step(20)
        a.adapt()
    img = a.checkpoint()
    from paper_2308_08085_gb300 import AmrLBM
    b = AmrLBM(cfg, storage="f32", use_graphs=False)
    b.restore(img)
    for sim in (a, b):
        sim.step(15)
        sim.adapt()
        sim.step(5)
    ca, cb = a.counts(), b.counts()
    ca.pop("launches")                      # kernels launched by each instance differ
    cb.pop("launches")
    assert ca == cb
    assert np.array_equal(a.nbr(), b.nbr())
    assert a.id_sets() == b.id_sets() and a.gaps() == b.gaps()
    assert np.array_equal(a.populations(), b.populations())
    c = new_gpu(W.cavity(dim=3, q=19, n=16, max_levels=2, max_blocks=64 * 20), "f32")
    from paper_2308_08085_gb300.amr import AmrError
    with pytest.raises(AmrError):
        c.restore(img)                      # other level count: refused
    for sim in (a, b, c):
        sim.close()



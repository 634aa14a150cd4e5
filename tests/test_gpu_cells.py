"""GPU parity of the cell-based uniform solver (the cell arrangement of the
comparison of cell- and block-based grids, Section 5) against the oracle's
dense uniform grid: periodic boxes of odd extents (several 256-thread tiles
and a ragged last tile), every velocity set, every element arrangement; at
the comparison's own size (192^3, D3Q19) the four arrangements agree bit for
bit and sampled cells match a per-cell oracle step.  FP32 bar: relative L2
<= 1e-5 against the FP64 oracle started from the FP32-rounded state."""
import numpy as np
import pytest

import workloads as W
from cellwise import CELL_TOL
from oracle.lattice import VelocitySet, bgk_collide, equilibrium, tau_level
from oracle.uniform import UniformLBM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def to_positions(a):
    """Array indexed [x, y(, z), p] -> [n, p] in x-fastest position order."""
    axes = tuple(range(a.ndim - 2, -1, -1)) + (a.ndim - 1,)
    return a.transpose(axes).reshape(-1, a.shape[-1])


def random_state(vs, shape, seed):
    n = int(np.prod(shape))
    rho, u = W.random_macro(seed, n, vs.dim)
    f = equilibrium(vs, rho, u) + W.random_noise(seed + 1, (n, vs.q), 1e-3)
    # the GPU starts from the FP32 rounding of this state; so does the oracle
    return f.astype(np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(2, 9, [37, 29]), (3, 19, [13, 11, 9]), (3, 27, [9, 10, 11])]
NU0 = 0.02


@pytest.mark.parametrize("arrangement", W.CELL_ARRANGEMENTS)
@pytest.mark.parametrize("dim,q,shape", CASES, ids=["d2q9", "d3q19", "d3q27"])
def test_cells_match_uniform_oracle(dim, q, shape, arrangement):
    from paper_2308_08085_gb300 import Cells
    vs = VelocitySet(dim, q)
    f0 = random_state(vs, shape, 41)                      # [n, q], x-fastest positions
    faces = [("periodic", (0.0, 0.0, 0.0))] * (2 * dim)
    ref = UniformLBM(dim, q, shape, tau_level(NU0, 0), faces)
    # x-fastest positions -> array indexed [x, y(, z)]
    ref.f = f0.reshape(tuple(reversed(shape)) + (q,)).transpose(
        tuple(range(dim - 1, -1, -1)) + (dim,)).copy()
    assert np.array_equal(to_positions(ref.f), f0)
    sim = Cells(dim, q, shape, NU0, W.cell_ids(shape, arrangement, seed=7))
    sim.set_f(f0)
    done = 0
    for k in (1, 2, 4):                                   # odd and even step counts
        sim.step(k)
        for _ in range(k):
            ref.step()
        done += k
        got = sim.f()
        want = to_positions(ref.f)
        err = rel_l2(got, want)
        assert err < TOL_F32, (arrangement, done, err)
        # worst cell (a uniform periodic grid has interior cells only)
        cell = np.max(np.abs(got - want) / np.maximum(np.abs(want), vs.w[None, :]))
        assert cell <= CELL_TOL["f32"], (arrangement, done, cell)


def test_cells_full_size_arrangements_agree_and_sampled_cells():
    """192^3 D3Q19 (the comparison's 3D size): every arrangement gives the same
    populations bit for bit after 3 steps (the per-cell arithmetic does not
    depend on the numbering), and 256 sampled cells after one step equal the
    oracle's collision of their upstream neighbours."""
    from paper_2308_08085_gb300 import Cells
    dim, q, shape = 3, 19, [192, 192, 192]
    vs = VelocitySet(dim, q)
    n = int(np.prod(shape))
    g = np.random.default_rng(5)
    # a smooth random flow: a few Fourier modes of rho and u plus noise
    pos = W.grid_positions(shape).astype(np.float64)
    ang = 2 * np.pi * pos / np.array(shape)
    rho = 1.0 + 0.01 * np.sin(ang[:, 0] + 2 * ang[:, 1]) * np.cos(ang[:, 2])
    u = 0.03 * np.stack([np.sin(ang[:, 1] + ang[:, 2]), np.cos(ang[:, 0] - ang[:, 2]),
                         np.sin(2 * ang[:, 0] + ang[:, 1])], 1)
    f0 = (equilibrium(vs, rho, u) + 1e-4 * (2 * g.random((n, q)) - 1)).astype(np.float32)
    del pos, ang, rho, u
    results = {}
    for arrangement in W.CELL_ARRANGEMENTS:
        sim = Cells(dim, q, shape, NU0, W.cell_ids(shape, arrangement, seed=11))
        sim.set_f(f0)
        sim.step(1)
        if arrangement == "calculated":
            one = sim.f()
        sim.step(2)
        results[arrangement] = sim.f()
        del sim
        torch.cuda.empty_cache()
    base = results["calculated"]
    for arrangement, got in results.items():
        assert np.array_equal(got, base), arrangement
    # sampled cells of the first step: f_p(x) = f*_p(x - c_p)
    idx = np.sort(g.choice(n, 256, replace=False))
    coords = W.grid_positions(shape)[idx]
    omega = 1.0 / tau_level(NU0, 0)
    want = np.empty((len(idx), q))
    for p in range(q):
        up = (coords - vs.c[p]) % np.array(shape)
        j = up[:, 0] + shape[0] * (up[:, 1] + shape[1] * up[:, 2])
        fstar, _, _ = bgk_collide(vs, f0[j].astype(np.float64), omega)
        want[:, p] = fstar[:, p]
    assert rel_l2(one[idx].astype(np.float64), want) < TOL_F32

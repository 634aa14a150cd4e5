"""GPU checks of the learned refinement proposal against the oracle: block
summaries, MLP gradient and inference, training progress, the dry-run
criterion, and the merging of proposal and criterion marks."""
import numpy as np
import pytest

import workloads as W
from oracle import learned as LN
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_08085_gb300 import build as b
    b.build()


def two_level(storage="f64"):
    from paper_2308_08085_gb300 import AmrLBM
    cfg = W.cavity(dim=3, q=19, n=12, ny=8, nz=8, max_levels=3, max_blocks=12 * 40)
    ref = ForestLBM(cfg)
    gpu = AmrLBM(cfg, storage=storage)
    m = np.zeros(cfg["max_blocks"], np.int8)
    m[[1, 2, 5, 6]] = 1
    ref.adapt(m)
    gpu.adapt(torch.from_numpy(m).cuda())
    ids = np.array(ref.mesh.active_ids())
    n = len(ids) * 64
    rho, u = W.random_macro(91, n, 3, drho=0.02, umax=0.04)
    f = equilibrium(ref.vs, rho, u) + W.random_noise(92, (n, 19), 5e-4)
    ref.f[ids] = f.reshape(len(ids), 64, 19)
    gpu.set_populations(ref.f)
    return cfg, ref, gpu


def test_block_features_match_oracle():
    cfg, ref, gpu = two_level()
    ref.step(2)
    gpu.step(2)
    ref.sync()
    got = gpu.features().cpu().numpy()
    for b in ref.mesh.active_ids():
        want = LN.block_features(ref, b)
        assert np.allclose(got[b], want, rtol=1e-4, atol=1e-4), (b, got[b] - want)
    gpu.close()


def test_mlp_gradient_and_inference_match_oracle():
    from paper_2308_08085_gb300 import Mlp
    dev = torch.device("cuda", 0)
    net = Mlp(dev, seed=7)
    g = np.random.default_rng(11)
    x = g.standard_normal((300, LN.IN)).astype(np.float32)
    y = (g.random(300) < 0.3).astype(np.float32)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    grad, loss = net.grad_of(xt, yt, pos_weight=2.0)
    p32 = net.params.cpu().numpy().astype(np.float64)
    l_ref, g_ref = LN.loss_and_grad(p32, x.astype(np.float64), y.astype(np.float64), 2.0)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    gg = grad.cpu().numpy()
    assert np.linalg.norm(gg - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    prob = net.infer(xt).cpu().numpy()
    ph = net.half.cpu().numpy().astype(np.float64)      # the FP16 weights inference reads
    _, p_ref = LN.forward(ph, x.astype(np.float64))
    assert np.max(np.abs(prob - p_ref)) <= 1e-5


def test_mlp_training_reduces_loss():
    from paper_2308_08085_gb300 import Mlp
    dev = torch.device("cuda", 0)
    net = Mlp(dev, seed=1)
    g = np.random.default_rng(5)
    x = g.standard_normal((4096, LN.IN)).astype(np.float32)
    y = ((x[:, 0] + 0.5 * x[:, 3]) > 0.3).astype(np.float32)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    first = net.train_epoch(xt, yt, batch=256, lr=3e-3, seed=0)
    for e in range(1, 8):
        last = net.train_epoch(xt, yt, batch=256, lr=3e-3, seed=e)
    assert last < 0.5 * first
    acc = ((net.infer(xt) > 0.5).float() == yt).float().mean().item()
    assert acc > 0.9


def test_dry_run_criterion_matches_oracle_and_merge():
    from paper_2308_08085_gb300 import Mlp
    cfg = W.channel_cylinder(q=19, nx=48, ny=24, nz=8, side=4, cx=16, cy=12, max_levels=3,
                             max_blocks=72 * 30, refine_dist=0.15)
    from paper_2308_08085_gb300 import AmrLBM
    ref = ForestLBM(cfg)
    gpu = AmrLBM(cfg, storage="f64")
    for _ in range(2):
        ref.step(10)
        gpu.step(10)
        ref.adapt()
        gpu.adapt()
    ref.step(10)
    gpu.step(10)
    ref.sync()
    want, _ = ref.criterion_marks()
    got = gpu.criterion_marks().cpu().numpy()
    assert np.array_equal(got, want)
    net = Mlp(torch.device("cuda", 0), seed=3)
    every = gpu.propose_marks(net.half, threshold=-1.0).cpu().numpy()   # p > -1: every leaf
    leaves = [b for b in ref.mesh.active_ids() if ref.mesh.status[b] == 1]
    assert np.all(every[leaves] >= 1)
    assert np.array_equal(every[every <= 0], want[every <= 0])
    none = gpu.propose_marks(net.half, threshold=2.0).cpu().numpy()      # p > 2: none
    assert np.array_equal(none, want)
    alone = gpu.propose_marks(net.half, threshold=2.0, with_criterion=False).cpu().numpy()
    assert not np.any(alone)
    gpu.close()

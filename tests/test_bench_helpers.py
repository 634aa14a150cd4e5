"""Host-side helpers of the benchmark: the sinusoid fit of the Strouhal
workload and the centreline sampling of the FP32/FP64 comparison, checked on
synthetic signals and on an oracle forest (no GPU)."""
import os
import sys

import numpy as np

import workloads as W
from oracle.lattice import equilibrium
from oracle.solver import ForestLBM

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fit_sinusoid_recovers_frequency_amplitude_and_mean():
    t = np.arange(8000, 16000, 16.0)
    for period, amp, mean in ((1067.0, 0.31, -0.004), (640.0, 1.2, 0.5)):
        g = np.random.default_rng(3)
        y = amp * np.sin(2 * np.pi * t / period + 0.7) + mean + 0.01 * g.standard_normal(len(t))
        f, a, m = bench.fit_sinusoid(t, y)
        assert abs(f * period - 1.0) < 2e-3
        assert abs(a - amp) < 0.01 * amp + 0.005
        assert abs(m - mean) < 0.005


class _Forest:
    """The attributes of AmrLBM that the centreline sampling reads, served
    from an oracle forest."""

    def __init__(self, lbm):
        self.lbm, self.cfg = lbm, lbm.cfg

    def rho_u(self):
        return self.lbm.macroscopic()

    def blocks(self):
        return dict(level=self.lbm.mesh.level, status=self.lbm.mesh.status)

    def coords(self):
        return self.lbm.mesh.X


def test_centreline_profiles_sample_the_leaf_cells():
    cfg = W.cavity(dim=3, q=19, n=16, max_levels=2, max_blocks=64 * 10)
    lbm = ForestLBM(cfg)
    m = np.zeros(cfg["max_blocks"], np.int8)
    m[[5, 6, 9, 10, 21, 22, 25, 26]] = 1
    lbm.adapt(m)
    for b in lbm.mesh.active_ids():
        x = lbm.cell_centres(b)
        u = np.stack([0.01 * x[:, 2], 0.0 * x[:, 0], 0.02 * x[:, 0]], 1)
        lbm.f[b] = equilibrium(lbm.vs, np.ones(len(x)), u)
    vx, vz = bench.centreline_profiles(_Forest(lbm), 32)
    s = (np.arange(32) + 0.5) * 16 / 32
    # each sample is the value at the centre of the leaf cell that holds it:
    # within half a cell of the sample point (half a root cell at most)
    assert np.all(np.abs(vx - 0.01 * s) <= 0.01 * 0.5 + 1e-12)
    assert np.all(np.abs(vz - 0.02 * s) <= 0.02 * 0.5 + 1e-12)
    assert np.all(np.diff(vx) >= -1e-12) and np.all(np.diff(vz) >= -1e-12)


def test_ncu_traffic_figure_matches_the_kernel_source():
    """The DRAM traffic per update that the bench line reports was captured by
    ncu on the kernel source with this hash; after a change to the kernel the
    figure is stale (the bench then reports null) until it is captured again."""
    assert bench.kernel_source_sha() == bench.NCU_SOURCE_SHA, (
        "collide-stream source changed: capture its DRAM traffic again and update "
        "NCU_TRAFFIC_PER_UPDATE / NCU_SOURCE_SHA")


def test_oracle_aggregate_and_cpu_info():
    """All-core oracle figure: every worker's updates over the longest
    worker's time, from the first counted step on."""
    res = [{"steps": [[10.0, 1.0, 1], [20.0, 2.0, 2]]},
           {"steps": [[30.0, 3.0, 3], [40.0, 4.0, 4]]}]
    v, u, s = bench.aggregate(res)
    assert u == 100.0 and s == 7.0 and abs(v - 100.0 / 7.0 / 1e6) < 1e-18
    v, u, s = bench.aggregate(res, first_step=1)
    assert u == 60.0 and s == 4.0
    info = bench.cpu_info()
    assert info["nproc"] == os.cpu_count() and info["machine"]


def test_oracle_sample_spins_up_and_times_whole_coarse_steps():
    s = bench.OracleSample(n=16)
    assert s.ups == s.sim.updates_per_coarse_step() > 0
    u, t, n = s.run(0.0)                 # at least one coarse step
    assert n == 1 and u == s.ups and t > 0
    assert "16^3" in s.describe()

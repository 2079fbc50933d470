"""The synthetic inputs follow their stated recipe: seeded and reproducible,
noise within its bounds around the inflow, Bingham numbers as defined for the
sphere study (Bi = tau0 D / (mu U), D = 2r), the sweep's parameters in range."""
import numpy as np
import pytest

from paper_1905_07392_gb300 import workloads as W


def test_initial_velocity_seeded_and_bounded():
    w = W.Workload("t", n=12, radius=0.2, seed=5, noise=1e-3)
    u1, u2 = W.initial_velocity(w), W.initial_velocity(w)
    assert u1.shape == (3, 12, 12, 12)
    assert np.array_equal(u1, u2)                                   # same seed, same input
    assert not np.array_equal(u1, W.initial_velocity(W.Workload("t", n=12, radius=0.2, seed=6)))
    for q in range(3):
        dev = u1[q] - w.u_in[q]
        assert np.abs(dev).max() <= w.noise
        assert abs(dev.mean()) < 5 * w.noise / np.sqrt(dev.size)   # centred noise
    f = W.body_force(w)
    assert np.array_equal(f, W.body_force(w)) and abs(f.std() - 0.1) < 0.01


def test_bingham_number_and_headline_workload():
    w = W.sphere_channel_256()
    assert (w.n, w.radius, w.m) == (256, 0.1, 1e4)
    assert w.bingham == pytest.approx(10.0, rel=1e-14)
    assert W.tau0_for_bingham(10.0, 0.1) == pytest.approx(50.0)
    assert w.bc == W.CHANNEL_BC and w.u_in == (0.0, 0.0, 1.0)


def test_batched_sweep_ranges():
    ws = W.batched_sweep(seed=0)
    assert len(ws) == 64 and ws == W.batched_sweep(seed=0)
    for w in ws:
        assert w.n in (48, 64, 96)
        assert 0.08 <= w.radius <= 0.2
        assert all(abs(c - 0.5) <= 0.05 for c in w.centre)
        assert 0.1 <= w.bingham <= 100.0 + 1e-9
    assert len({w.seed for w in ws}) == 64                          # independent noise per instance

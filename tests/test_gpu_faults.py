"""Failure statuses, made on the host (nothing here faults, traps or hangs the
GPU): a NaN in the velocity ends the step's solves with EBV_ERR_NAN (their
loops stop on a non-finite residual) and the context steps normally from a
good state afterwards; degenerate geometry gives EBV_ERR_GEOMETRY; an
allocation past the budget of ebv_set_alloc_limit gives EBV_ERR_OOM with
nothing left allocated; a wait of the fused smoother sweep on its tile loads
that runs out (ebv_set_spin_limit(0): every wait gives up at once, after
which the kernel lets its loads land and returns) gives EBV_ERR_TIMEOUT and
the context steps normally afterwards.  Also the step statistics: the
relative divergence and the per-phase GPU times of an eager step.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


def _channel(E, n=16, **kw):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    w.n = n
    s = E.Solver.from_workload(w, tol=1e-10, max_iters=500, **kw)
    alpha = s.geometry()["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=DEV) * (alpha > 0)).reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    return s, u, p, alpha


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_velocity_reports_nan_and_the_context_recovers(E, precision):
    s, u, p, alpha = _channel(E, precision=precision)
    good_u, good_p = u.clone(), p.clone()
    fluid = torch.nonzero(alpha > 0).flatten()
    u[2 * s.ncell + int(fluid[len(fluid) // 2])] = float("nan")
    with pytest.raises(E.EbvError) as ei:
        s.advance(u, p)
    assert ei.value.status == -5
    # the same context steps normally from a good state
    st = s.advance(good_u, good_p)
    assert max(st["res"]) <= 1e-10
    assert torch.isfinite(good_u).all()
    s.close()


def test_geometry_errors(E):
    n = 16
    s = E.Solver((n, n, n), 1.0 / n, tol=1e-10, tau0=1.0, m=1e3, bi_cfl=0.25)
    u = torch.zeros(3 * n ** 3, dtype=torch.float64, device=DEV)
    p = torch.zeros((n + 1) ** 3, dtype=torch.float64, device=DEV)
    with pytest.raises(E.EbvError) as ei:            # no geometry yet
        s.advance(u, p)
    assert ei.value.status == -6
    with pytest.raises(E.EbvError) as ei:            # the body covers the whole box
        s.build_sphere((0.5, 0.5, 0.5), 5.0)
    assert ei.value.status == -6
    s.close()
    # a box with no outflow side needs fluid at its pressure reference point
    s2 = E.Solver((n, n, n), 1.0 / n, bc=(E.INFLOW,) * 6, tol=1e-10, tau0=1.0, m=1e3, bi_cfl=0.25)
    with pytest.raises(E.EbvError) as ei:
        s2.build_sphere((0.0, 0.0, 0.0), 0.3)
    assert ei.value.status == -6
    s2.build_sphere((0.5, 0.5, 0.5), 0.2)           # fluid there: accepted
    s2.close()


def test_allocation_budget_gives_oom_and_nothing_leaks(E):
    lib = E.load()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.ebv_set_alloc_limit(1 << 20)                 # 1 MiB: far below a 32^3 context
    try:
        with pytest.raises(E.EbvError) as ei:
            E.Solver((32, 32, 32), 1.0 / 32, tol=1e-10)
        assert ei.value.status == -8
    finally:
        lib.ebv_set_alloc_limit(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    s, u, p, _ = _channel(E)                          # and a context works again
    assert max(s.advance(u, p)["res"]) <= 1e-10
    s.close()


def test_smoother_wait_limit_gives_timeout(E):
    lib = E.load()
    s, u, p, _ = _channel(E, n=32, precision=1)      # FP32 levels: 32^3 is smoothed by the fused sweep
    good_u, good_p = u.clone(), p.clone()
    lib.ebv_set_spin_limit(0)
    try:
        with pytest.raises(E.EbvError) as ei:
            s.advance(u, p)
        assert ei.value.status == -4
    finally:
        lib.ebv_set_spin_limit(-1)
    st = s.advance(good_u, good_p)
    assert max(st["res"]) <= 1e-10
    assert torch.isfinite(good_u).all()
    s.close()


def test_step_statistics(E):
    s, u, p, _ = _channel(E)
    st = s.advance(u, p)
    assert st["div_rel"] == max(st["res"][0], st["res"][4], st["res"][5], st["res"][9])
    assert 0.0 < st["div_rel"] <= 1e-10
    ms = st["ms"]
    assert all(v > 0.0 for v in ms.values()), ms
    # the viscous solves and projections dominate a step
    solve = ms["predictor_viscous"] + ms["corrector_viscous"] + ms["predictor_projection"] + \
        ms["corrector_projection"]
    assert solve > 0.3 * sum(ms.values())
    stg = s.advance_graph(u, p, steps=1)              # graph form: residuals, no phase times
    assert stg["div_rel"] == max(stg["res"][0], stg["res"][4], stg["res"][5], stg["res"][9])
    s.close()

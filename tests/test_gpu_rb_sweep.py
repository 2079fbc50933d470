"""The fused red-black sweep (one pass per Gauss-Seidel sweep, its tiles
staged in shared memory by TMA loads) against the pairs of colour passes it
replaces (paper Sec. "Numerical algorithm": red-black Gauss-Seidel smoothing
in the multigrid solves).  Whole FP32-refinement steps run with
ebv_set_fused_sweep(2) (always the fused sweep) and (0) (always the colour
passes) must give the same velocity, pressure and
solver statistics bit for bit, eager and as a captured graph: on the sphere
channel at 64^3 (levels 64, 32 fused) and on a box whose sizes are not
multiples of the 64 x 16 tile (80 x 40 x 48: ragged tiles in x and y, the
40-cell level below takes the colour passes in both runs).  Also the two
process-wide solver controls beside it: the set-up timings that choose the
sweep form (ebv_sweep_timing) and the inner drop of the refinement
(ebv_set_inner_drop), which must not change the tolerance the solves meet.
"""
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


def _run(E, shape, fused, graph, steps=3):
    import numpy as np
    from paper_1905_07392_gb300 import workloads as W
    lib = E.load()
    lib.ebv_set_fused_sweep(2 if fused else 0)
    try:
        w = W.sphere_channel_32()
        n = (shape,) * 3 if isinstance(shape, int) else tuple(shape)
        s = E.Solver(n, 1.0 / n[0], bc=w.bc, u_in=w.u_in, rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m,
                     model=w.model, bi_cfl=w.bingham, tol=1e-8, max_iters=500, precision=E.FP32_REFINE)
        s.build_sphere((0.5, 0.25, 0.3), 0.125)
        alpha = s.geometry()["alpha"]
        rng = np.random.Generator(np.random.PCG64(7))
        u0 = rng.uniform(-1e-3, 1e-3, size=(3, n[2] * n[1] * n[0]))
        u0[2] += 1.0
        u = (torch.tensor(u0, device=DEV) * (alpha > 0)).reshape(-1).contiguous()
        p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
        if graph:
            st = s.advance_graph(u, p, steps=steps)
        else:
            for _ in range(steps):
                st = s.advance(u, p)
        torch.cuda.synchronize()
        s.close()
        return u, p, st
    finally:
        lib.ebv_set_fused_sweep(1)


@pytest.mark.parametrize("shape", [64, (80, 40, 48)])
@pytest.mark.parametrize("graph", [False, True])
def test_fused_sweep_equals_colour_passes(E, shape, graph):
    u1, p1, st1 = _run(E, shape, True, graph)
    u0, p0, st0 = _run(E, shape, False, graph)
    assert torch.isfinite(u1).all() and torch.isfinite(p1).all()
    assert max(st1["res"]) <= 1e-8
    assert torch.equal(u1, u0)
    assert torch.equal(p1, p0)
    assert st1["iters"] == st0["iters"] and st1["res"] == st0["res"]


def test_sweep_timing_reported(E):
    """ebv_sweep_timing: once a step has run, each kind of sweep on the 64^3
    level (from zero, plain, after the coarse correction, with r.z) carries
    the set-up timings of both forms; a level or kind out of range is
    EBV_ERR_INVALID."""
    import numpy as np
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    n = (64, 64, 64)
    s = E.Solver(n, 1.0 / n[0], bc=w.bc, u_in=w.u_in, rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m,
                 model=w.model, bi_cfl=w.bingham, tol=1e-8, max_iters=500, precision=E.FP32_REFINE)
    try:
        s.build_sphere((0.5, 0.25, 0.3), 0.125)
        alpha = s.geometry()["alpha"]
        u0 = np.zeros((3, n[0] * n[1] * n[2]))
        u0[2] += 1.0
        u = (torch.tensor(u0, device=DEV) * (alpha > 0)).reshape(-1).contiguous()
        p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
        s.advance(u, p)
        torch.cuda.synchronize()
        for kind in range(4):
            f, q = s.sweep_timing(0, kind)
            assert 0.0 < f < 1e29 and 0.0 < q < 1e29, (kind, f, q)
        for lv, kind in ((99, 0), (0, 4), (-1, 0)):
            with pytest.raises(E.EbvError):
                s.sweep_timing(lv, kind)
    finally:
        s.close()


def test_inner_drop_keeps_tolerance(E):
    """ebv_set_inner_drop changes how far each FP32 correction of the
    refinement goes, not what the solves meet: steps run with drops 1e-2 and
    1e-6 both reach tol = 1e-11 in every solve and agree to 1e-8."""
    import numpy as np
    from paper_1905_07392_gb300 import workloads as W
    lib = E.load()
    out = []
    try:
        for drop in (1e-2, 1e-6):
            lib.ebv_set_inner_drop(drop)
            w = W.sphere_channel_32()
            n = (32, 32, 32)
            s = E.Solver(n, 1.0 / n[0], bc=w.bc, u_in=w.u_in, rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m,
                         model=w.model, bi_cfl=w.bingham, tol=1e-11, max_iters=2000,
                         precision=E.FP32_REFINE)
            s.build_sphere((0.5, 0.25, 0.3), 0.125)
            alpha = s.geometry()["alpha"]
            rng = np.random.Generator(np.random.PCG64(3))
            u0 = rng.uniform(-1e-3, 1e-3, size=(3, n[0] * n[1] * n[2]))
            u0[2] += 1.0
            u = (torch.tensor(u0, device=DEV) * (alpha > 0)).reshape(-1).contiguous()
            p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
            for _ in range(2):
                st = s.advance(u, p)
            torch.cuda.synchronize()
            s.close()
            assert max(st["res"]) <= 1e-11, (drop, st["res"])
            out.append(u.clone())
    finally:
        lib.ebv_set_inner_drop(-1.0)
    rel = ((out[0] - out[1]).norm() / out[1].norm()).item()
    assert rel <= 1e-8, rel

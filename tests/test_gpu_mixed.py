"""The precision form EBV_FP32_MIXED (paper Sec. "Strain rate tensor and
apparent viscosity", Algorithm 1): the strain rate and apparent viscosity of
fluid cells away from the EB are formed in FP32 from FP64 velocity
differences, those of cut cells and their neighbours in FP64.

* One viscosity update on the sphere channel at 64^3: cut cells (0 < alpha
  < 1) get the FP64 values bit for bit; every cell is within 1e-5 relative of
  the FP64 viscosity (FP32 norm, square root and viscosity law: a few FP32
  ulps, 6e-8 each; the Papanastasiou law divides by the strain rate, which
  can lift a few ulps of the rate to a few more of the viscosity).
* Five whole steps against the FP64 GPU path from the same seeded state:
  velocity within 1e-7 and pressure within 1e-6 relative (L2), drag within
  1e-7.  The viscosity error (~1e-6 relative at worst) enters only through
  the viscous increment of each step, itself a small part of u (noise of
  1e-3 on a uniform inflow; CFL-limited steps), so u moves by far less; the
  FP32_REFINE form itself sits at ~1e-10 (u) and ~4e-8 (p) from FP64.
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


def _state(E, precision, n=64):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    w.n = n
    s = E.Solver.from_workload(w, tol=1e-10, max_iters=2000, precision=precision)
    alpha = s.geometry()["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=DEV) * (alpha > 0)).reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    return s, u, p, alpha


def test_mixed_viscosity_update(E):
    s64, u, _, alpha = _state(E, E.FP64)
    sm, _, _, _ = _state(E, E.FP32_MIXED)
    e64 = torch.empty(s64.ncell, dtype=torch.float64, device=DEV)
    em = torch.empty_like(e64)
    s64.update_viscosity(u, e64)
    sm.update_viscosity(u, em)
    cut = (alpha > 0) & (alpha < 1)
    assert int(cut.sum()) > 0
    assert torch.equal(em[cut], e64[cut])
    fluid = alpha > 0
    rel = ((em - e64).abs() / e64.abs().clamp_min(1e-300))[fluid]
    assert float(rel.max()) <= 1e-5, float(rel.max())
    assert float(rel.max()) > 0.0          # the interior did take the FP32 path
    s64.close()
    sm.close()


def test_mixed_steps_against_fp64(E):
    runs = {}
    for prec in (E.FP64, E.FP32_MIXED):
        s, u, p, _ = _state(E, prec)
        dt = s.timestep(u)
        for _ in range(5):
            st = s.advance(u, p, dt=dt)
        runs[prec] = (u, p, st["drag"])
        s.close()
    (u0, p0, d0), (u1, p1, d1) = runs[E.FP64], runs[E.FP32_MIXED]
    ru = float(torch.linalg.vector_norm(u1 - u0) / torch.linalg.vector_norm(u0))
    rp = float(torch.linalg.vector_norm(p1 - p0) / torch.linalg.vector_norm(p0))
    assert ru <= 1e-7, ru
    assert rp <= 1e-6, rp
    assert abs(d1 - d0) <= 1e-7 * abs(d0), (d0, d1)

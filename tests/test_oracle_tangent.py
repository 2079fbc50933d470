"""Pins of the oracle's own derivatives (og_drag_tangent): forward-mode dual
numbers through the whole step of Algorithm 1 at a fixed time step, for the
drag of Eq. drag-force averaged over the steps.

- the value part is the double run, bit for bit (same operations, same order);
- d/dtau0 and d/dmu agree with central differences of the double oracle
  (the full step with the convective term, Bingham);
- a Newtonian creeping-flow step is affine in the body force f, and so is the
  drag (linear in u and p when eta = mu): any difference quotient along df is
  then exact, and the dual derivative must equal it to round-off;
- forward mode is linear in the direction: the derivative along
  (a dtau0, b dmu, df) is the same combination of the three separate ones.
"""
import numpy as np
import pytest

N, STEPS = 16, 3


def _case(O, model=None, advect=1, tau0=None):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    w.n = N
    g = O.Grid(n=(N, N, N), h=1.0 / N)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (w.radius,)))
    fl = geo.alpha > 0
    u0 = (W.initial_velocity(w).reshape(3, -1) * fl).ravel()
    rng = np.random.default_rng(3)
    f = (rng.normal(0.0, 0.1, (3, g.ncell)) * fl).ravel()
    df = (rng.normal(0.0, 1.0, (3, g.ncell)) * fl).ravel()
    P = O.Params(tau0=w.tau0 if tau0 is None else tau0, m=w.m, bi_cfl=w.bingham, tol=1e-13,
                 model=w.model if model is None else model, advect=advect)
    dt = O.timestep(g, geo, P, u0, f)
    return g, geo, P, u0, np.zeros(g.nnode), f, df, dt


def _J(O, g, geo, P, u0, p0, f, dt):
    u, p, acc = u0.copy(), p0.copy(), 0.0
    for _ in range(STEPS):
        u, p, st = O.advance(g, geo, P, u, p, dt=dt, f=f)
        acc += st["drag"]
    return acc / STEPS


def test_value_part_is_the_double_run(O):
    g, geo, P, u0, p0, f, df, dt = _case(O)
    J, _ = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, dtau0=1.0)
    assert J == _J(O, g, geo, P, u0, p0, f, dt)


def test_parameter_derivatives_match_central_differences(O):
    g, geo, P, u0, p0, f, df, dt = _case(O)
    for name, kw in (("tau0", {"dtau0": 1.0}), ("mu", {"dmu": 1.0})):
        _, dJ = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, **kw)
        x = getattr(P, name)
        h = 1e-5 * x

        def J_at(v):
            Q = O.Params(**{**P.__dict__, name: v})
            return _J(O, g, geo, Q, u0, p0, f, dt)

        fd = (J_at(x + h) - J_at(x - h)) / (2 * h)
        assert dJ == pytest.approx(fd, rel=1e-7), (name, dJ, fd)


def test_newtonian_creeping_drag_is_affine_in_the_force(O):
    g, geo, P, u0, p0, f, df, dt = _case(O, model=O.NEWTONIAN, advect=0, tau0=0.0)
    _, dJ = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, df=df)
    fd = (_J(O, g, geo, P, u0, p0, f + df, dt) - _J(O, g, geo, P, u0, p0, f - df, dt)) / 2.0
    assert abs(dJ) > 1e-8
    assert dJ == pytest.approx(fd, rel=1e-9), (dJ, fd)


def test_derivative_is_linear_in_the_direction(O):
    g, geo, P, u0, p0, f, df, dt = _case(O)
    _, dt0 = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, dtau0=1.0)
    _, dmu = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, dmu=1.0)
    _, dff = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, df=df)
    _, dall = O.drag_tangent(g, geo, P, u0, p0, dt, STEPS, f=f, df=df, dtau0=0.7, dmu=-1.3)
    comb = 0.7 * dt0 - 1.3 * dmu + dff
    assert dall == pytest.approx(comb, rel=1e-12, abs=1e-14 * (abs(dt0) + abs(dmu)))

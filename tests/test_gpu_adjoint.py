"""Adjoint of the step (ebv_adjoint_step / ebv_drag_gradient), in both forms:
creeping flow (advect = 0) and with the convective term (advect = 1): drag
sensitivities with respect to the yield stress, the plastic viscosity and a
per-cell body force, checked against central finite differences of the same
forward on the GPU (forward solves converged to 1e-13, so the difference
quotient is accurate to ~1e-7) and of the FP64 oracle's forward, and against
the oracle's own exact derivatives (forward-mode dual numbers, 1e-8).  Sphere
channel, Bingham (Bi = 5, m = 1e3), fixed dt from the CFL limit of the
initial state, checkpointing every 2 steps.  With the convective term the
limiter and the upwinding are piecewise linear: the seeded noise of the
initial state keeps their decisions away from ties (a uniform flow would sit
on the limiter's kink in every cell), so no kink lies within a difference
step.  The reverse kernels scatter with plain additions in a fixed order (no
atomics), so the gradients of two runs agree bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
N, R, STEPS, EVERY = 16, 0.2, 4, 2


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)
TOL_FD = 1e-5


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


def _setup(E, precision, newtonian=False, advect=0):
    from paper_1905_07392_gb300 import workloads as W
    w = W.Workload("adjoint_small", n=N, radius=R, tau0=W.tau0_for_bingham(5.0, R), m=1e3, seed=17)
    if newtonian:
        w = W.Workload("adjoint_small_newtonian", n=N, radius=R, tau0=0.0, model=W.NEWTONIAN, seed=17)
    s = E.Solver.from_workload(w, precision=precision, tol=1e-13, max_iters=20000, advect=advect)
    alpha = s.geometry()["alpha"]
    fluid = (alpha > 0).to(torch.float64)
    u0 = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=DEV) * fluid).reshape(-1).contiguous()
    p0 = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    f = (torch.tensor(W.body_force(w).reshape(3, -1), device=DEV) * fluid).reshape(-1).contiguous()
    dt = s.timestep(u0, f)
    return w, s, u0, p0, f, dt, fluid


def _objective(s, u0, p0, f, dt, steps=STEPS):
    u, p = u0.clone(), p0.clone()
    J = 0.0
    for _ in range(steps):
        J += s.advance(u, p, dt=dt, f=f, stats=True)["drag"]
    return J / steps


def _fd(fun, x, h):
    return (fun(x + h) - fun(x - h)) / (2 * h)


@pytest.mark.parametrize("precision,advect", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_drag_gradient_matches_finite_differences(E, precision, advect):
    w, s, u0, p0, f, dt, fluid = _setup(E, precision, advect=advect)
    J, gt, gm, fb = s.drag_gradient(u0, p0, dt, STEPS, EVERY, f=f)
    assert J == pytest.approx(_objective(s, u0, p0, f, dt), rel=1e-12)
    tau0, mu = s.params["tau0"], s.params["mu"]

    def J_tau(t):
        s.set_params(tau0=t)
        v = _objective(s, u0, p0, f, dt)
        s.set_params(tau0=tau0)
        return v

    def J_mu(m):
        s.set_params(mu=m)
        v = _objective(s, u0, p0, f, dt)
        s.set_params(mu=mu)
        return v

    fd_t = _fd(J_tau, tau0, 1e-6 * tau0)
    fd_m = _fd(J_mu, mu, 1e-6 * mu)
    assert abs(gt - fd_t) <= TOL_FD * abs(fd_t), (gt, fd_t)
    assert abs(gm - fd_m) <= TOL_FD * abs(fd_m), (gm, fd_m)
    # body force: directional derivative along a seeded field
    g = torch.Generator(device="cpu").manual_seed(5)
    d = (torch.randn(3 * s.ncell, generator=g, dtype=torch.float64).to(DEV) * fluid.repeat(3))
    eps = 1e-4
    fd_f = (_objective(s, u0, p0, f + eps * d, dt) - _objective(s, u0, p0, f - eps * d, dt)) / (2 * eps)
    ad_f = float(torch.dot(fb, d))
    assert abs(ad_f - fd_f) <= TOL_FD * abs(fd_f), (ad_f, fd_f)
    # f acts through psi only on fluid cells
    assert float(fb[fluid.repeat(3) == 0].abs().max()) == 0.0


def test_checkpointing_does_not_change_the_gradient(E):
    w, s, u0, p0, f, dt, fluid = _setup(E, 0)
    outs = [s.drag_gradient(u0, p0, dt, STEPS, every, f=f) for every in (1, 3, STEPS)]
    for J, gt, gm, fb in outs[1:]:
        assert J == outs[0][0]
        assert gt == pytest.approx(outs[0][1], rel=1e-12)
        assert gm == pytest.approx(outs[0][2], rel=1e-12)
        assert float((fb - outs[0][3]).abs().max()) <= 1e-12 * float(outs[0][3].abs().max())


@pytest.mark.parametrize("newtonian,advect,eps,tol", [(True, 0, 1e-3, 1e-9), (False, 0, 1e-7, 1e-5),
                                                     (False, 1, 1e-7, 1e-5)])
def test_single_step_adjoint_is_the_transpose(E, newtonian, advect, eps, tol):
    """<w, dS(u) du> = <S'(u)^T w, du>: the reverse pass of one step against a
    central difference of the forward step along a seeded perturbation of
    the initial velocity.  Newtonian: the creeping step is affine in u, so
    the difference is exact up to the solves.  Bingham (m = 1e3): eta varies
    on strain rates of 1/m, so the step must move u by much less than h/m."""
    w, s, u0, p0, f, dt, fluid = _setup(E, 0, newtonian, advect)
    g = torch.Generator(device="cpu").manual_seed(9)
    du = torch.randn(3 * s.ncell, generator=g, dtype=torch.float64).to(DEV) * fluid.repeat(3)
    wu = torch.randn(3 * s.ncell, generator=g, dtype=torch.float64).to(DEV) * fluid.repeat(3)
    wp = torch.randn(s.nnode, generator=g, dtype=torch.float64).to(DEV) * 1e-3
    ub, pb = wu.clone(), wp.clone()
    s.adjoint_step(u0, p0, dt, ub, pb, f=f)

    def step(u):
        uu, pp = u.clone(), p0.clone()
        s.advance(uu, pp, dt=dt, f=f, stats=False)
        return uu, pp

    up, pp_ = step(u0 + eps * du)
    um, pm = step(u0 - eps * du)
    lhs = float(torch.dot(wu, (up - um) / (2 * eps)) + torch.dot(wp, (pp_ - pm) / (2 * eps)))
    rhs = float(torch.dot(ub, du))
    assert abs(lhs - rhs) <= tol * abs(lhs), (lhs, rhs)


def test_autograd_function(E):
    w, s, u0, p0, f, dt, fluid = _setup(E, 0)
    t0 = s.params["tau0"]
    tau0 = torch.tensor(1.5 * t0, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(s.params["mu"], dtype=torch.float64, requires_grad=True)
    fr = f.clone().requires_grad_(True)
    J = E.drag_objective(s, tau0, mu, fr, u0, p0, dt, STEPS, EVERY)
    J.backward()
    assert s.params["tau0"] == t0            # the solver keeps its own parameters
    s.set_params(tau0=1.5 * t0)
    J2, gt, gm, fb = s.drag_gradient(u0, p0, dt, STEPS, EVERY, f=f)
    s.set_params(tau0=t0)
    assert float(J.detach()) == J2
    assert float(tau0.grad) == pytest.approx(gt, rel=1e-12)
    assert float(mu.grad) == pytest.approx(gm, rel=1e-12)
    assert float((fr.grad - fb).abs().max()) <= 1e-12 * float(fb.abs().max())


@pytest.mark.parametrize("advect", [0, 1])
def test_gradient_matches_oracle_finite_differences(E, O, advect):
    """Against the FP64 oracle's own forward (same problem, same dt): central
    differences of its time-averaged drag in tau0 and mu."""
    w, s, u0, p0, f, dt, fluid = _setup(E, 0, advect=advect)
    J, gt, gm, _ = s.drag_gradient(u0, p0, dt, STEPS, EVERY, f=f, f_grad=False)
    g = O.Grid(n=(N, N, N), h=1.0 / N, bc=w.bc, u_in=w.u_in)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (R,)))
    u0h, fh = u0.cpu().numpy(), f.cpu().numpy()

    def J_o(tau0, mu):
        P = O.Params(rho=w.rho, mu=mu, tau0=tau0, m=w.m, model=w.model, bi_cfl=w.bingham, tol=1e-13,
                     max_iters=200000, advect=advect)
        u, p = u0h.copy(), np.zeros(g.nnode)
        acc = 0.0
        for _ in range(STEPS):
            u, p, st = O.advance(g, geo, P, u, p, dt=dt, f=fh)
            acc += st["drag"]
        return acc / STEPS

    t0, m0 = w.tau0, w.mu
    assert J_o(t0, m0) == pytest.approx(J, rel=1e-9)
    ht, hm = 1e-4 * t0, 1e-4 * m0
    fd_t = (J_o(t0 + ht, m0) - J_o(t0 - ht, m0)) / (2 * ht)
    fd_m = (J_o(t0, m0 + hm) - J_o(t0, m0 - hm)) / (2 * hm)
    assert abs(gt - fd_t) <= TOL_FD * abs(fd_t), (gt, fd_t)
    assert abs(gm - fd_m) <= TOL_FD * abs(fd_m), (gm, fd_m)


@pytest.fixture(scope="module")
def dual_case(O):
    """The adjoint configuration on a 32^3 copy (sphere r = 0.125, Bi = 5,
    m = 1e3, seeded Gaussian body force of sigma 0.1), 8 steps at the CFL
    step of the initial state: the oracle's forward-mode derivatives of the
    time-averaged drag along tau0, mu and a seeded body-force direction."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import workloads as W
    w = W.Workload("adjoint_32", n=32, radius=0.125, tau0=W.tau0_for_bingham(5.0, 0.125), m=1e3, seed=3)
    g = O.Grid(n=(32, 32, 32), h=1.0 / 32)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (w.radius,)))
    fl = geo.alpha > 0
    u0 = (W.initial_velocity(w).reshape(3, -1) * fl).ravel()
    f = (W.body_force(w).reshape(3, -1) * fl).ravel()
    df = (np.random.Generator(np.random.PCG64(77)).normal(0.0, 1.0, (3, g.ncell)) * fl).ravel()
    P = O.Params(rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m, model=w.model, bi_cfl=w.bingham, tol=1e-13)
    dt = O.timestep(g, geo, P, u0, f)
    p0 = np.zeros(g.nnode)
    steps = 8
    out = {}
    for key, kw in (("tau0", {"dtau0": 1.0}), ("mu", {"dmu": 1.0}), ("f", {"df": df})):
        out["J"], out[key] = O.drag_tangent(g, geo, P, u0, p0, dt, steps, f=f, **kw)
    return w, u0, f, df, dt, steps, out


@pytest.mark.parametrize("precision", [0, 1])
def test_drag_gradient_matches_dual_oracle(E, dual_case, precision):
    """dJ/dtau0, dJ/dmu and <dJ/df, df> of the GPU adjoint (ebv_drag_gradient,
    checkpoints every 4 steps, the step with the convective term) against the
    oracle's exact forward-mode derivatives, to 1e-8 relative."""
    w, u0, f, df, dt, steps, ref = dual_case
    s = E.Solver.from_workload(w, precision=precision, tol=1e-13, max_iters=20000, advect=1)
    uu, ff = _t(u0), _t(f)
    p0 = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    J, gt, gm, fb = s.drag_gradient(uu, p0, dt, steps, 4, f=ff)
    assert J == pytest.approx(ref["J"], rel=1e-9)
    assert gt == pytest.approx(ref["tau0"], rel=1e-8), (gt, ref["tau0"])
    assert gm == pytest.approx(ref["mu"], rel=1e-8), (gm, ref["mu"])
    gf = float(torch.dot(fb, _t(df)))
    assert gf == pytest.approx(ref["f"], rel=1e-8), (gf, ref["f"])


@pytest.mark.parametrize("advect", [0, 1])
def test_gradients_bitwise_reproducible(E, advect):
    w, s, u0, p0, f, dt, fluid = _setup(E, 0, advect=advect)
    runs = [s.drag_gradient(u0, p0, dt, STEPS, EVERY, f=f) for _ in range(2)]
    (J1, gt1, gm1, fb1), (J2, gt2, gm2, fb2) = runs
    assert J1 == J2 and gt1 == gt2 and gm1 == gm2
    assert torch.equal(fb1, fb2)
    s.close()

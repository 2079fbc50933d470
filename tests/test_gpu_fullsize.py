"""GPU parity at the benchmark's size and launch configuration: 256^3 sphere
channel (r = 0.1, Bi = 10, m = 1e4), FP32 smoother with FP64 refinement, solve
tolerance 1e-8.

The oracle cannot run whole steps at this size in test time, so it checks
what it can compute directly: the geometry and the fused strain-rate /
viscosity kernel element by element, the face states element by element, and
every linear solve through the relative residual of its own operator applied
to the GPU solution (plus the velocity update of the nodal projection element
by element).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
TOL = 1e-8


@pytest.fixture(scope="module")
def case(O):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc, workloads as W
    build_lib.build()
    w = W.sphere_channel_256()
    s = ebvisc.Solver.from_workload(w, precision=ebvisc.FP32_REFINE, tol=TOL, max_iters=2000)
    n = w.n
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (w.radius,)))
    P = O.Params(rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m, model=w.model, bi_cfl=w.bingham, tol=TOL)
    u0 = (W.initial_velocity(w).reshape(3, -1) * (geo.alpha > 0)).ravel()
    return s, g, geo, P, u0


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)


def test_geometry_256(case):
    s, g, geo, P, u0 = case
    G = {k: v.cpu().numpy() for k, v in s.geometry().items()}
    assert (G["flag"] == geo.flag).all()
    for k in ("alpha", "ax", "ay", "az", "area"):
        assert np.abs(G[k] - getattr(geo, k)).max() < 1e-12, k
    A3g, A3o = np.tile(G["area"], 3), np.tile(geo.area, 3)
    assert np.abs(G["nrm"] * A3g - geo.nrm * A3o).max() < 1e-12
    assert np.abs(G["bcen"] * A3g - geo.bcen * A3o).max() < 1e-11


def test_strain_rate_viscosity_256(case, O):
    s, g, geo, P, u0 = case
    eta_o, sr_o = O.strain_eta(g, geo, P, u0)
    eta = torch.empty(g.ncell, dtype=torch.float64, device=DEV)
    sr = torch.empty_like(eta)
    s.update_viscosity(_t(u0), eta, sr)
    eta, sr = eta.cpu().numpy(), sr.cpu().numpy()
    assert np.abs(sr - sr_o).max() <= 1e-12 * np.abs(sr_o).max()
    assert np.abs(eta - eta_o).max() <= 1e-12 * np.abs(eta_o).max()


def test_face_states_and_projection_solve_256(case, O):
    s, g, geo, P, u0 = case
    uf_o = O.face_states(g, geo, u0)
    nft = sum(g.nface(d) for d in range(3))
    uf = torch.empty(nft, dtype=torch.float64, device=DEV)
    s.face_states(_t(u0), uf)
    assert np.abs(uf.cpu().numpy() - uf_o).max() < 1e-14
    phi = torch.empty(g.ncell, dtype=torch.float64, device=DEV)
    it, res = s.solve_mac(uf, phi)
    assert res <= TOL
    # residual of the oracle's cell-centred projection operator
    co = O.mac_coeffs(g, geo)
    nf = [g.nface(d) for d in range(3)]
    A = [geo.ax, geo.ay, geo.az]
    U = np.split(uf_o, np.cumsum(nf)[:2])
    b = np.zeros(g.ncell)
    for d in range(3):
        F = (A[d] * U[d]).reshape(g.fshape(d))
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[2 - d] = slice(1, None)
        lo[2 - d] = slice(0, -1)
        b -= (F[tuple(hi)] - F[tuple(lo)]).ravel() / g.h
    b[geo.alpha == 0] = 0.0
    r = b - O.cc_apply(g, co, phi.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01 * TOL * np.linalg.norm(b)


def test_viscous_solve_256(case, O):
    s, g, geo, P, u0 = case
    eta_o, _ = O.strain_eta(g, geo, P, u0)
    dt = O.timestep(g, geo, P, u0)
    rng = np.random.default_rng(5)
    psi = ((u0.reshape(3, -1) + 0.01 * rng.normal(size=(3, g.ncell))) * (geo.alpha > 0)).ravel()
    ut = torch.empty(3 * g.ncell, dtype=torch.float64, device=DEV)
    st = s.solve_viscous(_t(eta_o), _t(psi), dt, ut)
    assert max(st["res"][1:4]) <= TOL
    ut = ut.cpu().numpy().reshape(3, -1)
    for q in range(3):
        co, rb = O.visc_coeffs(g, geo, P, eta_o, dt, q)
        b = np.where(geo.alpha > 0, geo.alpha * psi.reshape(3, -1)[q] + rb, 0.0)
        r = b - O.cc_apply(g, co, ut[q])
        assert np.linalg.norm(r) <= 1.01 * TOL * np.linalg.norm(b), q


def test_nodal_projection_256(case, O):
    s, g, geo, P, u0 = case
    rng = np.random.default_rng(6)
    ut0 = ((u0.reshape(3, -1) + 0.05 * rng.normal(size=(3, g.ncell))) * (geo.alpha > 0)).ravel()
    dt = 1e-7
    ut, p = _t(ut0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    st = s.solve_projection(ut, p, dt)
    assert st["res"][4] <= TOL
    p = p.cpu().numpy()
    coef = dt / P.rho
    rhs = O.nodal_rhs(g, geo, ut0)
    r = rhs - O.nodal_apply(g, geo, coef, p)
    assert np.linalg.norm(r) <= 1.01 * TOL * np.linalg.norm(rhs)
    u_o = ut0 - coef * O.cell_grad_p(g, p) * np.tile(geo.alpha > 0, 3)
    assert np.abs(ut.cpu().numpy() - u_o).max() <= 1e-12 * np.abs(u_o).max()


def test_full_step_256(case, O):
    s, g, geo, P, u0 = case
    u, p = _t(u0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    st = s.advance(u, p)
    assert st["dt"] == pytest.approx(O.timestep(g, geo, P, u0), rel=1e-12)
    assert max(st["res"]) <= TOL
    un = u.cpu().numpy().reshape(3, -1)
    assert np.isfinite(un).all() and (un[:, geo.alpha == 0] == 0).all()
    assert np.isfinite(st["drag"]) and 0.0 <= st["yield_frac"] <= 1.0


def test_explicit_terms_256(case, O):
    """The explicit terms of Algorithm 2 at 256^3: the viscous term V (Eq.
    explicit-viscous with the EB wall flux of Eq. dudn) element by element
    against the oracle's, from the same velocity and the oracle's eta; the
    convective term C through an identity that holds for any face velocity:
    sum alpha C h^3 equals minus the net flux through the box faces (interior
    faces cancel, the EB carries none, redistribution conserves), with the
    GPU's own projected face velocities (the oracle cannot run the 256^3
    projection solve in test time)."""
    s, g, geo, P, u0 = case
    N3 = g.ncell
    Cv = torch.empty(3 * N3, dtype=torch.float64, device=DEV)
    V = torch.empty(3 * N3, dtype=torch.float64, device=DEV)
    eta = torch.empty(N3, dtype=torch.float64, device=DEV)
    s.derived(_t(u0), Cv, eta, V)
    eta_o, _ = O.strain_eta(g, geo, P, u0)
    V_o = O.viscous_explicit(g, geo, P, u0, eta_o)
    assert np.abs(V.cpu().numpy() - V_o).max() <= 1e-10 * np.abs(V_o).max()
    # C: the face velocities derived used (face states, projection), recomputed
    nft = sum(g.nface(d) for d in range(3))
    uf = torch.empty(nft, dtype=torch.float64, device=DEV)
    s.face_states(_t(u0), uf)
    s.solve_mac(uf, torch.empty(N3, dtype=torch.float64, device=DEV))
    ufd = np.split(uf.cpu().numpy(), np.cumsum([g.nface(d) for d in range(3)])[:2])
    aps = [geo.ax, geo.ay, geo.az]
    uq = u0.reshape(3, *g.cshape())
    C = Cv.cpu().numpy().reshape(3, N3)
    for q in range(3):
        net = 0.0
        for d in range(3):
            a = aps[d].reshape(g.fshape(d))
            w = ufd[d].reshape(g.fshape(d))
            for hs in (0, 1):
                fi = [slice(None)] * 3
                fi[2 - d] = -1 if hs else 0
                state = (np.full(a[tuple(fi)].shape, g.u_in[q]) if g.bc[2 * d + hs] == O.INFLOW
                         else uq[q][tuple(fi)])
                net += (1.0 if hs else -1.0) * (a[tuple(fi)] * state * w[tuple(fi)]).sum()
        total = (geo.alpha * C[q]).sum() * g.h ** 3
        scale = np.abs(geo.alpha * C[q]).sum() * g.h ** 3 + abs(net) * g.h ** 2
        assert abs(total + net * g.h ** 2) <= 1e-12 * scale, (q, total, -net * g.h ** 2)

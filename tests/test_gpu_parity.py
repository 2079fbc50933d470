"""GPU parity: the CUDA library (through its C-ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: geometry and pointwise kernels agree to rounding (1e-12); every
linear solve is run to a relative residual of 1e-13 on both sides and the
solutions agree to 1e-10 in relative L2 (the FP64 bar), which also holds for
whole steps.  The FP32 smoother path keeps FP64 residuals, so it reaches the
same solutions at the same tolerance.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


DEV = "cuda:0"


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)


def _pair(E, O, n, centre=(0.5, 0.5, 0.5), r=0.125, plane=None, bc=None, u_in=(0, 0, 1),
          tol=1e-13, precision=0, **prm):
    bc = bc or (O.SLIP, O.SLIP, O.SLIP, O.SLIP, O.INFLOW, O.OUTFLOW)
    args = dict(rho=1.0, mu=1.0, tau0=1.0, m=1e3, n_flow=1.0, eta0=1e3, model=O.BINGHAM,
                cfl=0.5, bi_cfl=0.25, delta_min=0.01)
    args.update(prm)
    s = E.Solver((n, n, n), 1.0 / n, bc=bc, u_in=u_in, tol=tol, max_iters=5000,
                 precision=precision, **args)
    g = O.Grid(n=(n, n, n), h=1.0 / n, bc=bc, u_in=u_in)
    if plane is not None:
        s.build_plane(plane[:3], plane[3])
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_PLANE, p=tuple(plane)))
    else:
        s.build_sphere(centre, r)
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(centre) + (r,)))
    P = O.Params(tol=tol, max_iters=200000, **args)
    return s, g, geo, P


def _noisy_u(g, geo, seed=0, amp=1e-3):
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-amp, amp, size=(3, g.ncell))
    u[2] += 1.0
    return (u * (geo.alpha > 0)).ravel()


@pytest.mark.parametrize("kind", ["sphere", "plane"])
def test_geometry_matches_oracle(E, O, kind):
    if kind == "sphere":
        s, g, geo, P = _pair(E, O, 32, centre=(0.5, 0.47, 0.53), r=0.2)
    else:
        nv = np.array([0.3, -0.5, 0.81])
        nv /= np.linalg.norm(nv)
        s, g, geo, P = _pair(E, O, 24, plane=tuple(nv) + (0.45,))
    G = {k: v.cpu().numpy() for k, v in s.geometry().items()}
    assert (G["flag"] == geo.flag).all()
    for k in ("alpha", "ax", "ay", "az", "area"):
        assert np.abs(G[k] - getattr(geo, k)).max() < 1e-12, k
    # the unit normal and centroid of a sliver cell amplify the rounding of
    # its tiny area vector: compare area-weighted
    A_gpu, A_o = G["area"], geo.area
    assert np.abs(G["nrm"] * np.tile(A_gpu, 3) - geo.nrm * np.tile(A_o, 3)).max() < 1e-12
    assert np.abs(G["bcen"] * np.tile(A_gpu, 3) - geo.bcen * np.tile(A_o, 3)).max() < 1e-11


@pytest.mark.parametrize("model,extra", [(1, {}), (0, {}), (2, {"n_flow": 0.5}),
                                         (3, {"n_flow": 1.4}), (4, {"n_flow": 0.6})])
def test_strain_rate_and_viscosity(E, O, model, extra):
    s, g, geo, P = _pair(E, O, 32, centre=(0.5, 0.5, 0.45), r=0.17, model=model, tau0=2.0,
                         **extra)
    u = _noisy_u(g, geo, seed=model, amp=0.05)
    eta_o, sr_o = O.strain_eta(g, geo, P, u)
    eta = torch.empty(g.ncell, dtype=torch.float64, device=DEV)
    sr = torch.empty_like(eta)
    s.update_viscosity(_t(u), eta, sr)
    eta, sr = eta.cpu().numpy(), sr.cpu().numpy()
    assert np.abs(sr - sr_o).max() <= 1e-12 * np.abs(sr_o).max()
    assert np.abs(eta - eta_o).max() <= 1e-12 * np.abs(eta_o).max()


def test_face_states_and_mac_projection(E, O):
    s, g, geo, P = _pair(E, O, 32)
    u = _noisy_u(g, geo, seed=3, amp=0.1)
    uf_o = O.face_states(g, geo, u)
    nft = sum(g.nface(d) for d in range(3))
    uf = torch.empty(nft, dtype=torch.float64, device=DEV)
    s.face_states(_t(u), uf)
    assert np.abs(uf.cpu().numpy() - uf_o).max() < 1e-14
    ufp_o, phi_o, it_o, res_o = O.mac_project(g, geo, uf_o, tol=1e-13)
    phi = torch.empty(g.ncell, dtype=torch.float64, device=DEV)
    it, res = s.solve_mac(uf, phi)
    assert res <= 1e-13
    assert _rel(phi.cpu().numpy(), phi_o) < 1e-10
    assert _rel(uf.cpu().numpy(), ufp_o) < 1e-12


def test_derived_quantities(E, O):
    s, g, geo, P = _pair(E, O, 32)
    u = _noisy_u(g, geo, seed=5, amp=0.05)
    C_o, eta_o, V_o, _ = O.derived(g, geo, P, u)
    Cv = torch.empty(3 * g.ncell, dtype=torch.float64, device=DEV)
    V = torch.empty_like(Cv)
    eta = torch.empty(g.ncell, dtype=torch.float64, device=DEV)
    s.derived(_t(u), Cv, eta, V)
    assert _rel(eta.cpu().numpy(), eta_o) < 1e-13
    assert _rel(Cv.cpu().numpy(), C_o) < 1e-9
    assert _rel(V.cpu().numpy(), V_o) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_viscous_solve(E, O, precision):
    s, g, geo, P = _pair(E, O, 32, precision=precision)
    u = _noisy_u(g, geo, seed=7, amp=0.05)
    eta_o, _ = O.strain_eta(g, geo, P, u)
    rng = np.random.default_rng(1)
    psi = (rng.normal(size=(3, g.ncell)) * (geo.alpha > 0)).ravel()
    dt = O.timestep(g, geo, P, u)
    ut_o, it_o, res_o = O.viscous_solve(g, geo, P, eta_o, psi, dt)
    ut = torch.empty(3 * g.ncell, dtype=torch.float64, device=DEV)
    st = s.solve_viscous(_t(eta_o), _t(psi), dt, ut)
    assert max(st["res"][1:4]) <= 1e-13
    assert _rel(ut.cpu().numpy(), ut_o) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_nodal_projection(E, O, precision):
    s, g, geo, P = _pair(E, O, 32, precision=precision)
    rng = np.random.default_rng(2)
    ut0 = (rng.normal(size=(3, g.ncell)) * (geo.alpha > 0)).ravel()
    p0 = rng.normal(size=g.nnode) * 0.1
    dt = 1e-3
    u_o, p_o, it_o, res_o = O.nodal_project(g, geo, P, dt, ut0, p0)
    ut, p = _t(ut0), _t(p0)
    st = s.solve_projection(ut, p, dt)
    assert st["res"][4] <= 1e-13
    assert _rel(p.cpu().numpy(), p_o) < 1e-10
    assert _rel(ut.cpu().numpy(), u_o) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_advance_config1_ten_steps(E, O, precision):
    """The plain-method configuration in full: sphere channel 32^3 (r = 0.125,
    tau_y = 1, m = 1e3), ten CFL steps, every step against the oracle."""
    s, g, geo, P = _pair(E, O, 32, precision=precision)
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    u0 = (W.initial_velocity(w).reshape(3, -1) * (geo.alpha > 0)).ravel()
    uo, po = u0.copy(), np.zeros(g.nnode)
    u, p = _t(u0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    for step in range(w.steps):
        uo, po, sto = O.advance(g, geo, P, uo, po)
        st = s.advance(u, p)
        assert st["dt"] == pytest.approx(sto["dt"], rel=1e-12)
        assert max(st["res"]) <= 1e-13
        assert _rel(u.cpu().numpy(), uo) < 1e-10, step
        assert _rel(p.cpu().numpy(), po) < 1e-10, step
        assert st["drag"] == pytest.approx(sto["drag"], rel=1e-9)
        assert st["yield_frac"] == pytest.approx(sto["yield_frac"], abs=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("walls", ["slip", "noslip"])
def test_ragged_odd_bottom(E, O, precision, walls):
    """A box with unequal sides and a bottom level of odd size (24 x 24 x 48 -> 3 x 3 x 6), in both
    precisions (the FP32 multigrid's row-split levels of odd width, its BF16 faces, the partial
    tiles of the nodal plane march) and with slip walls (each velocity component's viscous
    operator has its own Dirichlet sides) or no-slip walls (all share them)."""
    n = (24, 24, 48)
    h = 1.0 / 24
    w = O.SLIP if walls == "slip" else O.NOSLIP
    bc = (w, w, w, w, O.INFLOW, O.OUTFLOW)
    s = E.Solver(n, h, bc=bc, tol=1e-13, max_iters=5000, tau0=1.0, m=1e3, bi_cfl=0.3, precision=precision)
    s.build_sphere((0.5, 0.5, 0.9), 0.15)
    g = O.Grid(n=n, h=h, bc=bc)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.9, 0.15)))
    P = O.Params(tau0=1.0, m=1e3, bi_cfl=0.3, tol=1e-13)
    u0 = _noisy_u(g, geo, seed=11)
    uo, po, sto = O.advance(g, geo, P, u0, np.zeros(g.nnode))
    u, p = _t(u0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    s.advance(u, p)
    assert _rel(u.cpu().numpy(), uo) < 1e-10
    assert _rel(p.cpu().numpy(), po) < 1e-10


def test_empty_box_uniform_flow(E, O):
    """No body: uniform inflow is steady on the GPU too."""
    n = 16
    s = E.Solver((n, n, n), 1.0 / n, tol=1e-13, tau0=1.0, m=1e3, bi_cfl=0.25)
    s.build_geometry(lambda x: 1.0)
    u = torch.zeros(3 * n ** 3, dtype=torch.float64, device=DEV)
    u[2 * n ** 3:] = 1.0
    p = torch.zeros((n + 1) ** 3, dtype=torch.float64, device=DEV)
    st = s.advance(u, p)
    assert (u[2 * n ** 3:] - 1.0).abs().max().item() < 1e-13
    assert u[:2 * n ** 3].abs().max().item() < 1e-13
    assert p.abs().max().item() < 1e-10
    assert st["drag"] == 0.0


def test_host_buffer_step_matches_device_step(E, O):
    s, g, geo, P = _pair(E, O, 16, tol=1e-12)
    u0 = _noisy_u(g, geo, seed=4)
    uh, ph = u0.copy(), np.zeros(g.nnode)
    s.advance_host(uh, ph, 2)
    s2, *_ = _pair(E, O, 16, tol=1e-12)
    u, p = _t(u0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    s2.advance(u, p)
    s2.advance(u, p)
    assert np.array_equal(uh, u.cpu().numpy()) and np.array_equal(ph, p.cpu().numpy())


def test_reproducible_bitwise(E, O):
    s, g, geo, P = _pair(E, O, 16, tol=1e-10)
    u0 = _noisy_u(g, geo, seed=9)
    outs = []
    for _ in range(2):
        u, p = _t(u0), torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
        s.advance(u, p)
        outs.append((u.cpu().numpy(), p.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_errors_are_reported(E, O):
    s, g, geo, P = _pair(E, O, 16)
    u = torch.zeros(3 * g.ncell, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        s.advance(u[:-1], torch.zeros(g.nnode, dtype=torch.float64, device=DEV))
    with pytest.raises(E.EbvError):
        s.solve_viscous(torch.ones(g.ncell, dtype=torch.float64, device=DEV), u, -1.0, u.clone())
    s.set_params(max_iters=1, tol=1e-15)
    u2 = _t(_noisy_u(g, geo, seed=1, amp=0.3))
    with pytest.raises(E.EbvError) as ei:
        s.advance(u2, torch.zeros(g.nnode, dtype=torch.float64, device=DEV))
    assert ei.value.status == -3


@pytest.mark.parametrize("model", ["bingham", "herschel_bulkley"])
def test_flow_diagnostics(E, O, model):
    """Lambda of Eq. ryovar and the yield-stress deviation, cell by cell,
    on a sphere-cut 32^3 box with a seeded velocity field."""
    prm = {"model": O.HB, "n_flow": 0.5, "tau0": 2.0} if model == "herschel_bulkley" else {"tau0": 2.0}
    s, g, geo, P = _pair(E, O, 32, **prm)
    rng = np.random.default_rng(21)
    x = (np.arange(32) + 0.5) / 32
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.stack([np.sin(3 * Y) * Z, np.cos(2 * X) + 0.3 * Z, X * Y]) + 0.01 * rng.normal(size=(3, 32, 32, 32))
    u = (u.reshape(3, -1) * (geo.alpha > 0)).ravel()
    lam_o, dev_o = O.flow_diagnostics(g, geo, P, u)
    lam, dev = s.flow_diagnostics(_t(u))
    lam, dev = lam.cpu().numpy(), dev.cpu().numpy()
    assert np.abs(lam - lam_o).max() < 1e-10
    assert np.abs(dev - dev_o).max() <= 1e-12 * np.abs(dev_o).max()
    assert lam_o.min() < -0.5 and lam_o.max() > 0.5    # the field has rotation- and strain-dominated cells

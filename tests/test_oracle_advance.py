"""Pins of the oracle's whole step (Algorithm 1) and its reductions.

- Uniform inflow through an empty box is an exact steady state.
- A centred sphere in a noise-free channel keeps the mirror symmetries of the
  problem (x -> 1-x, y -> 1-y, x <-> y): catches transposed indices.
- Drag, pressure part: p = -z with u = 0 gives the buoyancy F_z = |body|
  (Eq. drag-force with the surface normal pointing into the fluid), O(h^2).
- Drag, viscous part: a plane wall with the Newtonian shear or extension flow
  u_z = gamma * (distance to the wall) and p = 0 has the traction
  mu gamma (1 + n_z^2) per unit wall area, which the wall-normal derivative
  of Eq. dudn reproduces exactly (it is exact on such fields): each term of
  the traction is checked by one wall orientation.
- Time step (Eqs. cfl:dt .. cfl:viscous:new): the classical limits.
"""
import numpy as np
import pytest


def test_uniform_flow_is_steady(O):
    n = 8
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    u = np.zeros((3, g.ncell))
    u[2] = 1.0
    P = O.Params(tau0=1.0, m=1e3, bi_cfl=0.25)
    u1, p1, st = O.advance(g, geo, P, u.ravel(), np.zeros(g.nnode))
    assert np.abs(u1 - u.ravel()).max() < 1e-13
    assert np.abs(p1).max() < 1e-10
    assert st["dt"] == pytest.approx(0.5 / (1.0 / g.h + 2 * 1.25 * 3 / g.h ** 2), rel=1e-14)


def test_sphere_channel_mirror_symmetry(O):
    # odd n: no face lies on a mirror plane, where the upwind choice of a
    # stationary shock (u_L = -u_R) would be decided by round-off
    n = 13
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.2)))
    u = np.zeros((3, g.ncell))
    u[2] = 1.0
    u *= geo.alpha > 0
    P = O.Params(tau0=1.0, m=1e3, bi_cfl=0.4, tol=1e-14)
    p = np.zeros(g.nnode)
    for _ in range(2):
        u, p, st = O.advance(g, geo, P, u.ravel(), p)
    U = u.reshape(3, n, n, n)  # (comp, z, y, x)
    scale = np.abs(U).max()
    tol = 1e-9 * scale
    assert np.abs(U[0] + U[0][:, :, ::-1]).max() < tol      # u_x odd in x
    assert np.abs(U[1] - U[1][:, :, ::-1]).max() < tol      # u_y even in x
    assert np.abs(U[2] - U[2][:, :, ::-1]).max() < tol
    assert np.abs(U[1] + U[1][:, ::-1, :]).max() < tol      # u_y odd in y
    assert np.abs(U[0] - U[1].transpose(0, 2, 1)).max() < tol  # x <-> y swap
    assert np.abs(U[2] - U[2].transpose(0, 2, 1)).max() < tol
    Pn = p.reshape(g.nshape())
    assert np.abs(Pn - Pn[:, :, ::-1]).max() < 1e-9 * np.abs(Pn).max()
    assert st["drag"] > 0


def test_buoyancy_drag_second_order(O):
    r = 0.2
    errs = []
    for n in (16, 32, 64):
        g = O.Grid(n=(n, n, n), h=1.0 / n)
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, r)))
        zn = np.meshgrid(*[np.arange(n + 1) * g.h] * 3, indexing="ij")[0]
        fz, yf = O.drag(g, geo, O.Params(tau0=1.0), np.zeros(3 * g.ncell), (-zn).ravel())
        errs.append(abs(fz - 4.0 / 3.0 * np.pi * r ** 3))
        assert yf == 1.0  # a fluid at rest is unyielded everywhere
    assert np.log2(errs[1] / errs[2]) > 1.5, errs


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_viscous_traction_drag_exact(O, axis):
    n = 16
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    x0 = 0.3 + 0.25 * g.h                       # inside a cell layer: one layer of cut cells
    nv = [0.0, 0.0, 0.0]
    nv[axis] = 1.0                              # fluid on the side x_axis > x0
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_PLANE, p=tuple(nv) + (x0,)))
    mu, gamma = 1.3, 0.7
    xc = (np.arange(n) + 0.5) * g.h
    coord = [np.broadcast_to(xc[None, None, :], (n, n, n)), np.broadcast_to(xc[None, :, None], (n, n, n)),
             np.broadcast_to(xc[:, None, None], (n, n, n))][axis].ravel()
    u = np.zeros((3, g.ncell))
    u[2] = np.where(geo.alpha > 0, gamma * (coord - x0), 0.0)
    P = O.Params(model=O.NEWTONIAN, mu=mu)
    fz, _ = O.drag(g, geo, P, u.ravel(), np.zeros(g.nnode))
    wall = geo.area.sum() * g.h ** 2
    assert wall == pytest.approx(1.0, rel=1e-12)  # the plane spans the unit cross-section
    nz2 = nv[2] ** 2
    assert fz == pytest.approx(mu * gamma * (1.0 + nz2) * wall, rel=1e-11)


def test_timestep_limits(O):
    n = 8
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    u = np.zeros((3, g.ncell))
    u[0, 5] = -3.0
    u[1, 5] = 2.0
    inviscid = O.Params(mu=0.0, cfl=0.5)
    assert O.timestep(g, geo, inviscid, u.ravel()) == pytest.approx(0.5 * g.h / 5.0, rel=1e-15)
    still = O.Params(mu=2.0, rho=3.0, bi_cfl=9.0, cfl=0.5)
    assert O.timestep(g, geo, still, 0 * u.ravel()) == pytest.approx(
        0.5 * 3.0 * g.h ** 2 / (2 * 2.0 * 10.0 * 3.0), rel=1e-15)
    f = np.zeros((3, g.ncell))
    f[2, 7] = 4.0
    forced = O.Params(mu=0.0, cfl=0.5)
    assert O.timestep(g, geo, forced, 0 * u.ravel(), f.ravel()) == pytest.approx(
        0.5 / np.sqrt(4.0 / g.h), rel=1e-14)


def test_creeping_newtonian_step_is_affine(O):
    """With C = 0 (creeping flow) and a Newtonian fluid the step at fixed dt
    is affine in (u, p, f): S(a x + (1 - a) y) = a S(x) + (1 - a) S(y).  The
    full step (advect = 1) is not (the convective term is quadratic): this
    pins that the switch removes exactly that term and nothing else."""
    n = 8
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.2)))
    rng = np.random.default_rng(3)
    fluid = np.tile(geo.alpha > 0, 3)
    xs = [((rng.normal(size=3 * g.ncell) + 0.3) * fluid, rng.normal(size=g.nnode),
           rng.normal(size=3 * g.ncell) * fluid) for _ in range(2)]
    a = 0.3
    mix = tuple(a * p + (1 - a) * q for p, q in zip(*xs))
    gaps = {}
    for advect in (0, 1):
        P = O.Params(model=O.NEWTONIAN, tau0=0.0, tol=1e-14, advect=advect)
        out = [O.advance(g, geo, P, u, p, dt=1e-3, f=f)[:2] for (u, p, f) in xs + [mix]]
        du = out[2][0] - (a * out[0][0] + (1 - a) * out[1][0])
        dp = out[2][1] - (a * out[0][1] + (1 - a) * out[1][1])
        gaps[advect] = max(np.abs(du).max() / np.abs(out[2][0]).max(), np.abs(dp).max() / np.abs(out[2][1]).max())
    assert gaps[0] < 1e-11
    assert gaps[1] > 1e-6


def test_taylor_green_between_slip_walls_second_order(O):
    """Whole step, time and space together (Sec. "Spatio-temporal convergence
    study: Taylor-Green vortices", Eq. taylor-green): the vortex at Re = 100
    between slip walls (the periodic solution satisfies them exactly) with
    the CFL step of Eqs. cfl:dt .. cfl:viscous:new to t = 0.25 (the last step
    shortened to end there); the velocity error at the cell centres falls at
    second order from 16^2 to 32^2 cells in the L1, L2 and max norms.  The box
    has no outflow side, so both pressure problems take the reference point
    (nodal p = 0 at node (0,0,0))."""
    from paper_1905_07392_gb300 import workloads as W
    errs = []
    for n in (16, 32):
        shape, h = W.taylor_green_grid(n)
        g = O.Grid(n=shape, h=h, bc=W.TG_BC, u_in=(0.0, 0.0, 0.0))
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
        P = O.Params(rho=1.0, mu=0.01, tau0=0.0, model=O.NEWTONIAN, tol=1e-12)
        u, p = W.taylor_green_velocity(n).ravel(), np.zeros(g.nnode)
        t = 0.0
        while t < 0.25 * (1.0 - 1e-12):
            dt = min(O.timestep(g, geo, P, u), 0.25 - t)
            u, p, st = O.advance(g, geo, P, u, p, dt=dt)
            t += dt
        assert p[0] == 0.0
        e = u.reshape(3, -1) - W.taylor_green_velocity(n, t=0.25).reshape(3, -1)
        mag = np.sqrt((e * e).sum(axis=0))
        errs.append((mag.mean(), np.sqrt((mag * mag).mean()), mag.max()))
        assert np.abs(u.reshape(3, -1)[2]).max() < 1e-10   # no flow out of the x-y plane
    rates = np.log2(np.array(errs[0]) / np.array(errs[1]))
    assert (rates > 1.8).all(), (errs, rates)


def test_uniform_flow_with_velocity_on_every_side_is_steady(O):
    """u = U e_z on every side (the paper's sphere and cylinder runs) around
    no body: uniform flow is an exact discrete solution; the pressure problems
    have no outflow side and take the reference point, so p stays 0."""
    n = 12
    g = O.Grid(n=(n, n, n), h=1.0 / n, bc=(O.INFLOW,) * 6, u_in=(0.0, 0.0, 1.0))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    P = O.Params(tau0=1.0, m=1e3, bi_cfl=1.0, tol=1e-13)
    u = np.concatenate([np.zeros(2 * g.ncell), np.ones(g.ncell)])
    u1, p1, st = O.advance(g, geo, P, u, np.zeros(g.nnode))
    assert np.abs(u1 - u).max() < 1e-12
    assert np.abs(p1).max() < 1e-12

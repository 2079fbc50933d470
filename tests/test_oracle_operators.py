"""Pins of the oracle's linear operators and solvers.

- Plane Poiseuille of a regularised Bingham fluid (Sec. "Convergence study for
  viscoplastic fluid", Eq. poiseuille:papabing, Appendix B): the steady
  discrete profile reproduces the paper's Table for z0 = 0 exactly and tracks
  it for z0 > 0.
- Symmetry of the alpha-weighted cell-centred and nodal operators.
- CG against a dense LU solve of the assembled matrix (small grids).
- Q1 nodal stiffness against Gauss quadrature of the trilinear basis.
- Manufactured solutions for the EB Dirichlet operator and the nodal
  projection; divergence after the cell-centred projection.
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lambert_w(x):
    w = np.log1p(x) if x < 3 else np.log(x) - np.log(np.log(x))
    for _ in range(200):
        ew = np.exp(w)
        f = w * ew - x
        dw = f / (ew * (w + 1) - (w + 2) * f / (2 * w + 2))
        w -= dw
        if abs(dw) < 1e-15 * (1 + abs(w)):
            break
    return w


def papanastasiou_poiseuille(z, z0, eps):
    """Eq. poiseuille:papabing (z0 = 0: the Newtonian parabola)."""
    z = np.abs(z)
    if z0 == 0:
        return 1 - z ** 2
    xi = 2 * z0 / (eps * (1 - z0) ** 2)
    W = np.vectorize(_lambert_w)
    return (1 - ((z - z0) / (1 - z0)) ** 2
            + z0 * eps / (2 * xi) * ((1 + W(xi * np.exp(-xi * (z / z0 - 1)))) ** 2
                                     - (1 + W(xi * np.exp(-xi * (1 / z0 - 1)))) ** 2))


def _centres(g):
    n = g.n
    z, y, x = np.meshgrid(*[g.lo[2 - q] + (np.arange(n[2 - q]) + 0.5) * g.h for q in range(3)],
                          indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _poiseuille_errors(O, N, z0, eps=0.01):
    """Steady plane Poiseuille: Picard iteration eta <- eta(u), solve
    -d/dz(eta du/dz) = G with no-slip walls at z = -1, 1 (dimensionless,
    mu = W = U = 1, tau0 = Bi = 2 z0 / (1 - z0)^2, G = 2 / (1 - z0)^2)."""
    h = 2.0 / N
    g = O.Grid(n=(2, 2, N), lo=(0, 0, -1), h=h,
               bc=(O.OUTFLOW, O.OUTFLOW, O.SLIP, O.SLIP, O.NOSLIP, O.NOSLIP), u_in=(0, 0, 0))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    bi = 2 * z0 / (1 - z0) ** 2
    P = O.Params(rho=0.0, mu=1.0, tau0=bi, m=1 / eps,
                 model=O.BINGHAM if z0 > 0 else O.NEWTONIAN)
    G = 2 / (1 - z0) ** 2
    zc = -1 + (np.arange(N) + 0.5) * h
    ue = papanastasiou_poiseuille(zc, z0, eps)
    u = np.zeros((3, N, 2, 2))
    u[0] = ue[:, None, None]
    for _ in range(400):
        eta, _ = O.strain_eta(g, geo, P, u.ravel())
        co, rb = O.visc_coeffs(g, geo, P, eta, 1.0, 0)
        x, _, _ = O.cc_solve(g, co, np.full(g.ncell, G) + rb, x0=u[0].ravel())
        change = np.abs(x - u[0].ravel()).max()
        u[0] = x.reshape(N, 2, 2)
        if change < 1e-13:
            break
    e = np.abs(u[0][:, 0, 0] - ue)
    return e.mean(), np.sqrt((e ** 2).mean()), e.max()


def _table():
    rows = {}
    for line in open(os.path.join(GOLDEN, "poiseuille_bingham_eps0.01.txt")):
        if line.strip() and not line.startswith("#"):
            z0, N, *v = line.split()
            rows[(float(z0), int(N))] = tuple(map(float, v))
    return rows


def test_poiseuille_newtonian_matches_table_exactly(O):
    tab = _table()
    for N in (16, 32, 64, 128):
        errs = _poiseuille_errors(O, N, 0.0)
        for mine, paper in zip(errs, tab[(0.0, N)]):
            assert mine == pytest.approx(paper, rel=1e-9)


@pytest.mark.parametrize("z0,rtol", [(0.1, 0.05), (0.2, 0.05), (0.5, 0.25)])
def test_poiseuille_bingham_tracks_table(O, z0, rtol):
    tab = _table()
    mine = {N: _poiseuille_errors(O, N, z0) for N in (16, 32, 64)}
    for N in (16, 32, 64):
        for a, b in zip(mine[N], tab[(z0, N)]):
            assert a == pytest.approx(b, rel=rtol), (z0, N, mine[N], tab[(z0, N)])
    # same convergence rate in every norm (within 0.15)
    for q in range(3):
        r_m = np.log2(mine[32][q] / mine[64][q])
        r_p = np.log2(tab[(z0, 32)][q] / tab[(z0, 64)][q])
        assert abs(r_m - r_p) < 0.15, (z0, q, r_m, r_p)


@pytest.fixture(scope="module")
def sphere16(O):
    g = O.Grid(n=(16, 16, 16), h=1.0 / 16)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.52, 0.47, 0.27)))
    return g, geo


def test_cc_operators_symmetric(O, sphere16):
    g, geo = sphere16
    rng = np.random.default_rng(1)
    eta = (1 + 100 * rng.random(g.ncell)) * (geo.alpha > 0)
    P = O.Params(rho=1.0)
    for comp in range(3):
        co, _ = O.visc_coeffs(g, geo, P, eta, 0.01, comp)
        x, y = rng.normal(size=(2, g.ncell))
        assert np.dot(O.cc_apply(g, co, x), y) == pytest.approx(np.dot(x, O.cc_apply(g, co, y)),
                                                                rel=1e-13)
    co = O.mac_coeffs(g, geo)
    x, y = rng.normal(size=(2, g.ncell))
    assert np.dot(O.cc_apply(g, co, x), y) == pytest.approx(np.dot(x, O.cc_apply(g, co, y)),
                                                            rel=1e-13)


def _assemble(apply, n):
    M = np.zeros((n, n))
    e = np.zeros(n)
    for q in range(n):
        e[q] = 1.0
        M[:, q] = apply(e)
        e[q] = 0.0
    return M


def test_cg_matches_dense_lu(O):
    g = O.Grid(n=(8, 8, 8), h=1.0 / 8)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.22)))
    rng = np.random.default_rng(2)
    eta = (1 + 1000 * rng.random(g.ncell)) * (geo.alpha > 0)
    P = O.Params(rho=1.0)
    co, _ = O.visc_coeffs(g, geo, P, eta, 1e-3, 2)
    M = _assemble(lambda v: O.cc_apply(g, co, v), g.ncell)
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    b = rng.normal(size=g.ncell)
    x, it, res = O.cc_solve(g, co, b, tol=1e-14)
    xd = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    coef = 0.37
    Mn = _assemble(lambda v: O.nodal_apply(g, geo, coef, v), g.nnode)
    assert np.allclose(Mn, Mn.T, rtol=0, atol=1e-13 * np.abs(Mn).max())
    bn = rng.normal(size=g.nnode)
    # identity rows (Dirichlet / isolated nodes) carry a zero right-hand side
    ident = np.isclose(np.diag(Mn), 1.0) & (np.abs(Mn).sum(axis=1) == 1.0)
    bn[ident] = 0.0
    p, it, res = O.nodal_solve(g, geo, coef, bn, tol=1e-14)
    pd = np.linalg.solve(Mn, bn)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)


def test_mac_operator_exact_on_quadratics_without_eb(O):
    n = 10
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    co = O.mac_coeffs(g, geo)
    x, y, z = _centres(g)
    phi = 1.0 + x - 2 * y + 3 * x * z + 0.5 * x * x - y * y + 2 * z * z
    lap = 1.0 - 2.0 + 4.0
    Aphi = O.cc_apply(g, co, phi).reshape(g.cshape())
    assert np.abs(Aphi[1:-1, 1:-1, 1:-1] + lap).max() < 1e-9


def _gauss_q1_stiffness():
    """int over [0,1]^3 of grad N_a . grad N_b, by 2-point Gauss quadrature."""
    gp = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    K = np.zeros((8, 8))
    for xq in itertools.product(gp, repeat=3):
        grads = []
        for o in range(8):
            bits = [(o >> d) & 1 for d in range(3)]
            val = [xq[d] if bits[d] else 1 - xq[d] for d in range(3)]
            der = [1.0 if bits[d] else -1.0 for d in range(3)]
            grads.append([der[d] * np.prod([val[e] for e in range(3) if e != d])
                          for d in range(3)])
        grads = np.array(grads)
        K += grads @ grads.T / 8.0
    return K


def test_nodal_stencil_is_q1_stiffness(O):
    n = 6
    h = 1.0 / n
    g = O.Grid(n=(n, n, n), h=h, bc=(O.SLIP,) * 6)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    K = _gauss_q1_stiffness()
    coef = 2.5
    p = np.zeros(g.nnode)
    c = (3, 3, 3)
    p[(c[2] * (n + 1) + c[1]) * (n + 1) + c[0]] = 1.0
    y = O.nodal_apply(g, geo, coef, p).reshape(g.nshape())
    # assemble the expected 27-point stencil from the element matrix
    exp = np.zeros((3, 3, 3))
    for cell in itertools.product((-1, 0), repeat=3):
        oa = sum(((-cell[d]) << d) for d in range(3))
        for ob in range(8):
            off = [cell[d] + ((ob >> d) & 1) for d in range(3)]
            exp[off[2] + 1, off[1] + 1, off[0] + 1] += K[ob, oa]
    got = y[c[2] - 1:c[2] + 2, c[1] - 1:c[1] + 2, c[0] - 1:c[0] + 2] / (coef * h)
    assert np.abs(got - exp).max() < 1e-13
    assert exp[1, 1, 1] == pytest.approx(8.0 / 3.0)


def test_nodal_uniform_inflow_is_solenoidal(O):
    n = 8
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    ut = np.zeros((3, g.ncell))
    ut[2] = 1.0
    r = O.nodal_rhs(g, geo, ut.ravel())
    assert np.abs(r).max() < 1e-15
    P = O.Params(rho=1.0)
    u, p, it, res = O.nodal_project(g, geo, P, 0.01, ut.ravel(), np.zeros(g.nnode))
    assert np.abs(p).max() < 1e-14 and np.abs(u - ut.ravel()).max() < 1e-14


def test_nodal_projection_removes_gradients(O):
    """u~ = grad q with q = 0 at the outflow: the projection returns u ~ 0
    and p ~ rho q / dt; the errors shrink under refinement."""
    errs_u, errs_p = [], []
    for n in (16, 32):
        g = O.Grid(n=(n, n, n), h=1.0 / n, bc=(O.SLIP, O.SLIP, O.SLIP, O.SLIP, O.NOSLIP, O.OUTFLOW))
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
        x, y, z = _centres(g)
        k = np.pi
        # q with zero normal derivative on the walls and q(z=1) = 0
        gq = np.stack([-k * np.sin(k * x) * np.cos(k * y) * np.cos(0.5 * k * z),
                       -k * np.cos(k * x) * np.sin(k * y) * np.cos(0.5 * k * z),
                       -0.5 * k * np.cos(k * x) * np.cos(k * y) * np.sin(0.5 * k * z)])
        dt, rho = 0.01, 1.0
        u, p, it, res = O.nodal_project(g, geo, O.Params(rho=rho), dt, gq.ravel(),
                                        np.zeros(g.nnode))
        zn, yn, xn = np.meshgrid(*[np.arange(n + 1) * g.h] * 3, indexing="ij")
        qn = np.cos(k * xn) * np.cos(k * yn) * np.cos(0.5 * k * zn)
        errs_u.append(np.abs(u).max())
        errs_p.append(np.abs(p.reshape(g.nshape()) * dt / rho - qn).max())
    assert errs_u[1] < 0.3 * errs_u[0] and errs_p[1] < 0.3 * errs_p[0], (errs_u, errs_p)


def test_mac_projection_divergence_free(O, sphere16):
    g, geo = sphere16
    rng = np.random.default_rng(4)
    u = (rng.normal(size=(3, g.ncell)) + np.array([[0], [0], [1.0]])) * (geo.alpha > 0)
    uf0 = O.face_states(g, geo, u.ravel())
    uf, phi, it, res = O.mac_project(g, geo, uf0, tol=1e-13)
    nf = [g.nface(d) for d in range(3)]
    A = [geo.ax, geo.ay, geo.az]
    U = np.split(uf, np.cumsum(nf)[:2])
    U0 = np.split(uf0, np.cumsum(nf)[:2])

    def div(U):
        s = 0
        for d in range(3):
            F = (A[d] * U[d]).reshape(g.fshape(d))
            sl_hi = [slice(None)] * 3
            sl_lo = [slice(None)] * 3
            sl_hi[2 - d] = slice(1, None)
            sl_lo[2 - d] = slice(0, -1)
            s = s + F[tuple(sl_hi)] - F[tuple(sl_lo)]
        return s.ravel()
    d0, d1 = div(U0), div(U)
    assert np.linalg.norm(d1) <= 1e-12 * np.linalg.norm(d0)
    # apertures of covered faces are zero; velocities on them are untouched zeros
    assert np.abs(uf[np.concatenate(A) == 0]).max() == 0.0


def test_eb_dirichlet_manufactured_rates(O):
    """Poisson with u = 0 on the sphere and the box: u = (|x-c|^2 - r^2) S(x).
    Measured orders of the face-centred EB operator with the wall distance
    bounded below at 0.01 cells: L1 1.73, Linf 0.99 (32 -> 64); pinned at
    L1 >= 1.6, Linf >= 0.9."""
    r = 0.2
    e1, einf = [], []
    for n in (16, 32, 64):
        g = O.Grid(n=(n, n, n), h=1.0 / n, bc=(O.NOSLIP,) * 6, u_in=(0, 0, 0))
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, r)))
        x, y, z = _centres(g)
        pi = np.pi
        S = np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
        f = (x - .5) ** 2 + (y - .5) ** 2 + (z - .5) ** 2 - r * r
        gS = [pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z),
              pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z),
              pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)]
        lap = 6 * S + 4 * ((x - .5) * gS[0] + (y - .5) * gS[1] + (z - .5) * gS[2]) \
            - 3 * pi ** 2 * f * S
        P = O.Params(rho=0.0, mu=1.0, model=O.NEWTONIAN)
        fl = geo.alpha > 0
        co, _ = O.visc_coeffs(g, geo, P, fl * 1.0, 1.0, 0)
        xs, it, res = O.cc_solve(g, co, np.where(fl, -geo.alpha * lap, 0.0))
        err = np.abs(xs - f * S)[fl]
        e1.append(err.mean())
        einf.append(err.max())
    assert np.log2(e1[1] / e1[2]) > 1.6 and np.log2(einf[1] / einf[2]) > 0.9, (e1, einf)

"""Pins of the oracle's pointwise and stencil parts.

- eta(||gamma_dot||) (Table "Generalised Newtonian fluid models"): limits and
  the paper's printed yield strain eps W(Bi/eps) = 0.010397 (Eq. lambertw).
- strain rate (Sec. "Strain rate tensor and apparent viscosity"): exact on
  quadratic fields wherever the central / one-sided quadratic stencils apply;
  simple shear gives ||gamma_dot|| = |gamma|.
- wall gradient (Eq. dudn): exact for a profile quadratic in the wall distance.
- slopes/upwinding, redistribution conservation (Eq. divergence_final),
  explicit viscous term by manufactured solutions.
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lambert_w(x):
    """Principal branch by Halley's iteration (Corless et al. 1996)."""
    w = np.log1p(x) if x < 3 else np.log(x) - np.log(np.log(x))
    for _ in range(100):
        ew = np.exp(w)
        f = w * ew - x
        dw = f / (ew * (w + 1) - (w + 2) * f / (2 * w + 2))
        w -= dw
        if abs(dw) < 1e-15 * (1 + abs(w)):
            break
    return w


def test_eta_limits(O):
    P = O.Params(mu=1.5, tau0=2.0, m=1e3, model=O.BINGHAM)
    assert O.eta_of(P, 0.0) == pytest.approx(1.5 + 2.0 * 1e3, rel=1e-15)
    assert O.eta_of(P, 1e-12) == pytest.approx(1.5 + 2.0 * 1e3, rel=1e-8)
    assert O.eta_of(P, 50.0) == pytest.approx(1.5 + 2.0 / 50.0, rel=1e-15)
    Pn = O.Params(mu=1.5, tau0=2.0, model=O.NEWTONIAN)
    assert O.eta_of(Pn, 3.0) == 1.5
    Ph = O.Params(mu=1.5, tau0=2.0, m=1e3, n_flow=1.0, model=O.HB)
    for s in (0.0, 1e-4, 0.3, 7.0):
        assert O.eta_of(Ph, s) == pytest.approx(O.eta_of(P, s), rel=1e-14)
    Ph5 = O.Params(mu=1.0, tau0=0.0, m=1e3, n_flow=0.5, model=O.HB)
    assert O.eta_of(Ph5, 4.0) == pytest.approx(0.5, rel=1e-14)
    assert O.eta_of(Ph5, 0.0) == pytest.approx(np.sqrt(1e3), rel=1e-14)  # floor 1/m


def test_eta_power_law_closed_values(O):
    """Power law (Table "Generalised Newtonian fluid models": kappa s^(n-1)),
    the OG_POWERLAW branch itself: closed values for n = 0.5 and n = 2, the
    floor s >= 1/m for n < 1, n = 1 is Newtonian, no yield term whatever tau0."""
    P = O.Params(mu=3.0, tau0=7.0, m=100.0, n_flow=0.5, model=O.POWERLAW)
    assert O.eta_of(P, 4.0) == pytest.approx(1.5, rel=1e-15)       # 3 / sqrt(4)
    assert O.eta_of(P, 0.25) == pytest.approx(6.0, rel=1e-15)      # 3 / sqrt(1/4)
    assert O.eta_of(P, 1e-6) == pytest.approx(30.0, rel=1e-15)     # floored at 1/m = 0.01
    assert O.eta_of(P, 0.0) == pytest.approx(30.0, rel=1e-15)
    P2 = O.Params(mu=3.0, tau0=7.0, m=100.0, n_flow=2.0, model=O.POWERLAW)
    for sr in (0.5, 2.0, 9.0):
        assert O.eta_of(P2, sr) == pytest.approx(3.0 * sr, rel=1e-15)   # shear thickening
    P1 = O.Params(mu=3.0, tau0=7.0, m=100.0, n_flow=1.0, model=O.POWERLAW)
    for sr in (0.0, 0.3, 5.0):
        assert O.eta_of(P1, sr) == pytest.approx(3.0, rel=1e-15)
    # log-slope (n - 1) between any two strain rates above the floor
    for sr in (0.05, 1.0, 40.0):
        r = np.log(O.eta_of(P, 2.0 * sr) / O.eta_of(P, sr)) / np.log(2.0)
        assert r == pytest.approx(-0.5, abs=1e-14)


def test_eta_souza_mendes_dutra_closed_values(O):
    """Souza Mendes-Dutra (Table "Generalised Newtonian fluid models":
    kappa s^(n-1) + tau0 (1 - exp(-eta0 s / tau0)) / s): a closed value at
    eta0 s / tau0 = 1, the s -> 0 limit kappa (1/m)^(n-1) + eta0, the
    large-s stress tau0 + kappa s^n, and the identity with the regularised
    Herschel-Bulkley law when eta0 = tau0 m."""
    P = O.Params(mu=1.0, tau0=2.0, eta0=4.0, m=1e3, n_flow=1.0, model=O.SMD)
    assert O.eta_of(P, 0.5) == pytest.approx(1.0 + 4.0 * (1.0 - np.exp(-1.0)), rel=1e-15)
    assert O.eta_of(P, 0.0) == pytest.approx(1.0 + 4.0, rel=1e-15)
    Pn = O.Params(mu=0.7, tau0=2.0, eta0=4.0, m=1e3, n_flow=0.5, model=O.SMD)
    assert O.eta_of(Pn, 0.0) == pytest.approx(0.7 * np.sqrt(1e3) + 4.0, rel=1e-14)
    sr = 1e4
    assert O.eta_of(Pn, sr) * sr == pytest.approx(2.0 + 0.7 * sr ** 0.5, rel=1e-15)
    for n in (0.5, 1.0, 1.6):
        Ps = O.Params(mu=0.7, tau0=2.0, eta0=2.0 * 250.0, m=250.0, n_flow=n, model=O.SMD)
        Ph = O.Params(mu=0.7, tau0=2.0, m=250.0, n_flow=n, model=O.HB)
        for s_ in (0.0, 1e-3, 0.02, 1.0, 30.0):
            assert O.eta_of(Ps, s_) == pytest.approx(O.eta_of(Ph, s_), rel=1e-14)


def test_yield_strain_printed_value(O):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "yield_strain.txt"))
            if l.strip() and not l.startswith("#")]
    bi, eps, printed = map(float, rows[0])
    s_star = eps * _lambert_w(bi / eps)
    assert round(s_star, 6) == pytest.approx(printed, abs=1e-6)
    # dimensionless (mu = U = D = 1, tau0 = Bi): the stress magnitude
    # eta(s) s reaches the yield stress exactly at s_star
    P = O.Params(mu=1.0, tau0=bi, m=1.0 / eps, model=O.BINGHAM)
    assert O.eta_of(P, s_star) * s_star == pytest.approx(bi, rel=1e-13)
    assert O.eta_of(P, 0.5 * s_star) * 0.5 * s_star < bi
    assert O.eta_of(P, 2.0 * s_star) * 2.0 * s_star > bi


def _avail_mask(g, geo):
    a = geo.alpha.reshape(g.cshape()) > 0
    return a


def _second_order_cells(g, geo):
    """Cells whose three 1-D stencils are central or one-sided quadratic."""
    a = _avail_mask(g, geo)
    nz, ny, nx = a.shape
    ok = a.copy()
    for ax in range(3):
        n = a.shape[ax]

        def sh(s):
            out = np.zeros_like(a)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if s > 0:
                src[ax], dst[ax] = slice(s, n), slice(0, n - s)
            else:
                src[ax], dst[ax] = slice(0, n + s), slice(-s, n)
            out[tuple(dst)] = a[tuple(src)]
            return out
        p1, m1, p2, m2 = sh(1), sh(-1), sh(2), sh(-2)
        good = (p1 & m1) | (~p1 & m1 & m2) | (p1 & ~m1 & p2)
        ok &= good
    return ok.ravel()


def _centres(g):
    n = g.n
    z, y, x = np.meshgrid(*[g.lo[2 - q] + (np.arange(n[2 - q]) + 0.5) * g.h for q in range(3)],
                          indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def test_strain_rate_exact_on_quadratics(O):
    n = 20
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.45, 0.55, 0.23)))
    x, y, z = _centres(g)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3))
    Q = rng.normal(size=(3, 3, 3))  # u_c = A_c.x + x^T Q_c x
    X = np.stack([x, y, z])
    u = np.stack([A[c] @ X + np.einsum("in,ij,jn->n", X, Q[c], X) for c in range(3)])
    # analytic G[d][c] = du_c/dx_d
    G = np.zeros((3, 3, x.size))
    for c in range(3):
        for d in range(3):
            G[d, c] = A[c, d] + (Q[c][d, :] + Q[c][:, d]) @ X
    gam = G + G.transpose(1, 0, 2)
    s_exact = np.sqrt(0.5 * (gam ** 2).sum(axis=(0, 1)))
    P = O.Params(mu=1.0, tau0=0.0, model=O.NEWTONIAN)
    u = u * (geo.alpha > 0)
    eta, sr = O.strain_eta(g, geo, P, u.ravel())
    ok = _second_order_cells(g, geo)
    assert ok.sum() > 0.9 * (geo.alpha > 0).sum()
    assert np.abs(sr[ok] - s_exact[ok]).max() < 1e-9 * np.abs(s_exact).max()
    Gn = O.cell_gradient(g, geo, u.ravel()).reshape(3, 3, -1)
    assert np.abs(Gn[:, :, ok] - G[:, :, ok]).max() < 1e-9 * np.abs(G).max()
    assert (sr[geo.alpha == 0] == 0).all() and (eta[geo.alpha == 0] == 0).all()


def test_simple_shear_norm(O):
    n = 16
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.2)))
    x, y, z = _centres(g)
    gam = 2.7
    u = np.stack([gam * z, 0 * z, 0 * z]) * (geo.alpha > 0)
    _, sr = O.strain_eta(g, geo, O.Params(model=O.NEWTONIAN), u.ravel())
    fl = geo.alpha > 0
    assert np.abs(sr[fl] - gam).max() < 1e-12


def test_wall_gradient_exact_for_quadratic_profile(O):
    nv = np.array([0.3, -0.5, 0.81])
    nv /= np.linalg.norm(nv)
    d = 0.45
    n = 24
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_PLANE, p=tuple(nv) + (d,)))
    x, y, z = _centres(g)
    s = nv[0] * x + nv[1] * y + nv[2] * z - d  # distance from the wall
    a_c = np.array([1.3, -0.7, 2.1])
    b_c = np.array([0.4, 3.0, -1.1])
    u = np.stack([a_c[q] * s + b_c[q] * s ** 2 for q in range(3)]) * (geo.alpha > 0)
    cut = np.nonzero(geo.flag == 2)[0]
    k, j, i = np.unravel_index(cut, g.cshape())
    interior = (i > 3) & (i < n - 4) & (j > 3) & (j < n - 4) & (k > 3) & (k < n - 4)
    checked = 0
    for c in cut[interior]:
        for q in range(3):
            val = O.wall_dudn(g, geo, u.ravel(), int(c), q)
            assert val == pytest.approx(a_c[q], rel=1e-9, abs=1e-9)
        checked += 1
    assert checked > 50


def test_slopes_and_upwind_linear_field(O):
    n = 12
    g = O.Grid(n=(n, n, n), h=1.0 / n, bc=(O.OUTFLOW,) * 6)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    x, y, z = _centres(g)
    u = np.stack([1.0 + 0.3 * x, 2.0 - 0.2 * y, 0.5 + 0.1 * z])
    uf = O.face_states(g, geo, u.ravel())
    ux = uf[:g.nface(0)].reshape(g.fshape(0))
    # faces between two interior cells: both extrapolations equal the face
    # value of a linear field (boundary cells carry zero slopes)
    xf = np.arange(2, n - 1) * g.h
    assert np.abs(ux[:, :, 2:n - 1] - (1.0 + 0.3 * xf)[None, None, :]).max() < 1e-13
    assert np.abs(ux[:, :, 1] - (1.0 + 0.3 * 0.5 * g.h)).max() < 1e-13
    # upwinding of the normal component (Godunov for Burgers)
    u2 = np.stack([np.where(x < 0.5, -1.0, 1.0), 0 * x, 0 * x])  # rarefaction -> 0
    uf2 = O.face_states(g, geo, u2.ravel())[:g.nface(0)].reshape(g.fshape(0))
    assert (uf2[:, :, n // 2] == 0).all()
    u3 = np.stack([np.where(x < 0.5, 2.0, -1.0), 0 * x, 0 * x])  # shock moving right -> uL
    uf3 = O.face_states(g, geo, u3.ravel())[:g.nface(0)].reshape(g.fshape(0))
    assert (uf3[:, :, n // 2] == 2.0).all()
    u4 = np.stack([np.where(x < 0.5, 1.0, -2.0), 0 * x, 0 * x])  # shock moving left -> uR
    uf4 = O.face_states(g, geo, u4.ravel())[:g.nface(0)].reshape(g.fshape(0))
    assert (uf4[:, :, n // 2] == -2.0).all()


def test_redistribution_conserves(O):
    n = 16
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.3)))
    rng = np.random.default_rng(0)
    DC = rng.normal(size=g.ncell) * (geo.alpha > 0)
    D = O.redistribute(g, geo, DC)
    a = geo.alpha
    assert abs((a * D).sum() - (a * DC).sum()) < 1e-12 * np.abs(a * DC).sum()
    far = geo.flag == 1
    # regular cells whose neighbourhood is regular keep D = D^C exactly
    f3 = (geo.flag.reshape(g.cshape()) == 1)
    allreg = f3.copy()
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        allreg &= np.roll(f3, (dz, dy, dx), axis=(0, 1, 2))
    allreg[[0, -1], :, :] = allreg[:, [0, -1], :] = allreg[:, :, [0, -1]] = False
    sel = allreg.ravel() & far
    assert sel.sum() > 100
    assert (D[sel] == DC[sel]).all()
    # small cells get a bounded update: D^H stays within neighbour range
    geo0 = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    assert (O.redistribute(g, geo0, DC * 0 + 1.0) == 1.0).all()


def test_explicit_viscous_manufactured(O):
    """V_j = div(eta grad(u)^T)_j for smooth u and eta, no EB: interior O(h^2)."""
    errs = []
    for n in (16, 32):
        g = O.Grid(n=(n, n, n), h=1.0 / n, bc=(O.OUTFLOW,) * 6)
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
        x, y, z = _centres(g)
        k = 2 * np.pi
        u = np.stack([np.sin(k * y) * np.cos(k * z) + x * y,
                      np.cos(k * x) * z, np.sin(k * x) * np.sin(k * y)])
        eta = 1.0 + 0.5 * np.sin(k * x) * np.cos(k * z)
        # analytic: V_j = sum_i d/dx_i (eta du_i/dx_j)
        dux = [[y, x + k * np.cos(k * y) * np.cos(k * z), -k * np.sin(k * y) * np.sin(k * z)],
               [-k * np.sin(k * x) * z, 0 * x, np.cos(k * x)],
               [k * np.cos(k * x) * np.sin(k * y), k * np.sin(k * x) * np.cos(k * y), 0 * x]]
        # du[i][j] = du_i/dx_j; need d/dx_i of eta du_i/dx_j
        deta = [0.5 * k * np.cos(k * x) * np.cos(k * z), 0 * x,
                -0.5 * k * np.sin(k * x) * np.sin(k * z)]
        # second derivatives d/dx_i (du_i/dx_j) = d/dx_j (div u); div u = y + 0 + 0
        ddiv = [0 * x, 1 + 0 * x, 0 * x]
        V = np.stack([sum(deta[i] * dux[i][j] for i in range(3)) + eta * ddiv[j]
                      for j in range(3)])
        P = O.Params(rho=1.0)
        Vn = O.viscous_explicit(g, geo, P, u.ravel(), eta).reshape(3, *g.cshape())
        Ve = V.reshape(3, *g.cshape())
        s = slice(2, n - 2)
        errs.append(np.abs(Vn[:, s, s, s] - Ve[:, s, s, s]).max())
    assert np.log2(errs[0] / errs[1]) > 1.8, errs

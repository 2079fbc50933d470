"""Pins of the oracle's convective term (Sec. "Convective term", Eqs.
divergence_conservative .. divergence_final with zero EB flux): C = -div(u (x) u^F).

- a velocity field linear in x, y, z on a box without EB: slope-limited face
  states are exact, so C equals -((A u)_q + u_q tr A) at every cell two or more
  cells from the box, to round-off;
- a step in u_q advected by a uniform face velocity: the limiter gives zero
  slopes and the upwind state is the upstream cell's value, so C is the
  first-order upwind difference, for either sign of the velocity;
- a smooth quadratic field: C converges at O(h^2) in the interior;
- a sphere-cut box with random u and u^F: sum alpha C h^3 equals minus the
  net flux through the box faces (interior faces cancel, the EB carries no
  flux, redistribution conserves), to round-off; the sphere also cuts a box
  face, so the box-face apertures enter;
- a uniform state U advected by a uniform face velocity W past a sphere: the
  face fluxes of a cut cell sum, by the divergence theorem, to the flux the
  closed EB face would carry, U_q (W . n) A / (alpha h), which the
  (separately pinned) redistribution then spreads: C = -redistribute(that).
"""
import numpy as np
import pytest


def _grid(O, n, bc=None):
    kw = {} if bc is None else {"bc": bc}
    return O.Grid(n=n, h=1.0 / max(n), **kw)


def _centres(g):
    nz, ny, nx = g.cshape()
    z, y, x = np.meshgrid(*[g.lo[d] + (np.arange(m) + 0.5) * g.h for d, m in ((2, nz), (1, ny), (0, nx))],
                          indexing="ij")
    return x, y, z


def _face_centres(g, d):
    shp = g.fshape(d)
    coords = []
    for e, m in ((2, shp[0]), (1, shp[1]), (0, shp[2])):
        off = 0.0 if e == d else 0.5
        coords.append(g.lo[e] + (np.arange(m) + off) * g.h)
    z, y, x = np.meshgrid(*coords, indexing="ij")
    return x, y, z


def _face_field(g, fn):
    """Face triple of the d-th velocity component fn(d, x, y, z) at face centres."""
    return np.concatenate([fn(d, *_face_centres(g, d)).ravel() for d in range(3)])


A = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.25, 0.2, 0.15]])
U0 = np.array([0.7, -0.4, 1.1])


def _lin(d, x, y, z):
    return U0[d] + A[d, 0] * x + A[d, 1] * y + A[d, 2] * z


def test_linear_field_exact(O):
    g = _grid(O, (10, 11, 12))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    x, y, z = _centres(g)
    u = np.concatenate([_lin(q, x, y, z).ravel() for q in range(3)])
    uf = _face_field(g, _lin)
    C = O.convective(g, geo, u, uf).reshape(3, *g.cshape())
    tr = np.trace(A)
    inner = (slice(2, -2),) * 3
    for q in range(3):
        Au = sum(A[q, d] * _lin(d, x, y, z) for d in range(3))
        exact = -(Au + _lin(q, x, y, z) * tr)
        err = np.abs(C[q][inner] - exact[inner]).max()
        assert err < 1e-12 * np.abs(exact[inner]).max(), (q, err)


@pytest.mark.parametrize("w", [0.8, -0.6])
def test_step_is_upwinded(O, w):
    n = (12, 6, 5)
    g = _grid(O, n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    nz, ny, nx = g.cshape()
    i = np.arange(nx)
    steps = [(4, 1.0), (6, 2.0), (3, 0.5)]  # jump position and height per component
    prof = [np.where(i >= i0, hgt, 0.0) for i0, hgt in steps]
    u = np.concatenate([np.broadcast_to(p_, (nz, ny, nx)).ravel() for p_ in prof])
    uf = np.concatenate([np.full(g.nface(0), w), np.zeros(g.nface(1)), np.zeros(g.nface(2))])
    C = O.convective(g, geo, u, uf).reshape(3, nz, ny, nx)
    for q, p_ in enumerate(prof):
        up = np.zeros(nx)
        for c in range(1, nx - 1):
            up[c] = (p_[c] - p_[c - 1]) if w > 0 else (p_[c + 1] - p_[c])
        exact = -w * up / g.h
        for c in range(1, nx - 1):
            assert np.allclose(C[q][:, :, c], exact[c], rtol=0, atol=1e-12), (q, c)


def _quad(d, x, y, z):
    # monotone in every direction on [0, 1]^3, so the MC limiter keeps the
    # central slope everywhere in the interior
    c = [(1.0, 0.5, 0.2, 0.1, 0.25), (-0.5, 0.2, 0.6, 0.3, 0.15), (0.8, 0.1, 0.3, 0.7, 0.2)][d]
    return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * (x * x + y * z)


def _quad_grad(d):
    c = [(1.0, 0.5, 0.2, 0.1, 0.25), (-0.5, 0.2, 0.6, 0.3, 0.15), (0.8, 0.1, 0.3, 0.7, 0.2)][d]
    return (lambda x, y, z: c[1] + 2 * c[4] * x,
            lambda x, y, z: c[2] + c[4] * z,
            lambda x, y, z: c[3] + c[4] * y)


def test_quadratic_field_second_order(O):
    errs = []
    for n in (16, 32, 64):
        g = _grid(O, (n, n, n))
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
        x, y, z = _centres(g)
        u = np.concatenate([_quad(q, x, y, z).ravel() for q in range(3)])
        C = O.convective(g, geo, u, _face_field(g, _quad)).reshape(3, n, n, n)
        box = (np.abs(x - 0.5) < 0.25) & (np.abs(y - 0.5) < 0.25) & (np.abs(z - 0.5) < 0.25)
        e = 0.0
        for q in range(3):
            exact = -sum(_quad_grad(q)[d](x, y, z) * _quad(d, x, y, z) +
                         _quad(q, x, y, z) * _quad_grad(d)[d](x, y, z) for d in range(3))
            e = max(e, np.abs(C[q] - exact)[box].max())
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > 1.8).all(), (errs, rates)


def test_sphere_cut_box_conserves(O):
    n = (14, 12, 16)
    g = _grid(O, n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.43, 0.09, 0.52, 0.23)))
    ay0 = geo.ay.reshape(g.fshape(1))[:, 0, :]
    assert ((ay0 > 0) & (ay0 < 1)).sum() > 5  # the y- box face is cut
    rng = np.random.default_rng(7)
    N3 = g.ncell
    fluid = geo.alpha > 0
    u = (rng.uniform(-1, 1, (3, N3)) * fluid).ravel()
    aps = [geo.ax, geo.ay, geo.az]
    uf = np.concatenate([rng.uniform(-1, 1, g.nface(d)) * (aps[d] > 0) for d in range(3)])
    # every open interior face separates two fluid cells (precondition of the
    # cancellation of interior fluxes)
    al = geo.alpha.reshape(g.cshape())
    for d in range(3):
        a = aps[d].reshape(g.fshape(d))
        sl = [slice(None)] * 3
        sl[2 - d] = slice(1, -1)
        lo = [slice(None)] * 3
        lo[2 - d] = slice(0, -1)
        hi = [slice(None)] * 3
        hi[2 - d] = slice(1, None)
        open_ = a[tuple(sl)] > 0
        assert (al[tuple(lo)][open_] > 0).all() and (al[tuple(hi)][open_] > 0).all()
    C = O.convective(g, geo, u, uf).reshape(3, N3)
    ufd = np.split(uf, [g.nface(0), g.nface(0) + g.nface(1)])
    uq = u.reshape(3, *g.cshape())
    for q in range(3):
        net = 0.0
        for d in range(3):
            a = aps[d].reshape(g.fshape(d))
            w = ufd[d].reshape(g.fshape(d))
            for hs in (0, 1):
                side = 2 * d + hs
                fi = [slice(None)] * 3
                fi[2 - d] = -1 if hs else 0
                ci = [slice(None)] * 3
                ci[2 - d] = -1 if hs else 0
                state = (np.full(a[tuple(fi)].shape, g.u_in[q]) if g.bc[side] == O.INFLOW
                         else uq[q][tuple(ci)])
                net += (1.0 if hs else -1.0) * (a[tuple(fi)] * state * w[tuple(fi)]).sum()
        total = (geo.alpha * C[q]).sum() * g.h ** 3
        assert total == pytest.approx(-net * g.h ** 2, abs=1e-13 * max(1.0, abs(net) * g.h ** 2)), q


def test_uniform_state_cut_cells(O):
    n = (14, 12, 16)
    U = np.array([0.3, -0.7, 1.2])
    Wv = np.array([0.4, 0.25, -0.9])
    g = O.Grid(n=n, h=1.0 / 16, u_in=tuple(U))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.43, 0.37, 0.52, 0.23)))
    N3 = g.ncell
    fluid = geo.alpha > 0
    cut = geo.flag == 2
    assert cut.sum() > 50
    u = (U[:, None] * fluid[None, :]).ravel()
    uf = np.concatenate([np.full(g.nface(d), Wv[d]) for d in range(3)])
    C = O.convective(g, geo, u, uf).reshape(3, N3)
    nrm = geo.nrm.reshape(3, N3)
    wn = (Wv[:, None] * nrm).sum(0)
    for q in range(3):
        DC = np.zeros(N3)
        DC[cut] = U[q] * wn[cut] * geo.area[cut] / (geo.alpha[cut] * g.h)
        exact = -O.redistribute(g, geo, DC)
        assert np.abs(C[q] - exact).max() < 1e-12 * np.abs(exact).max(), q

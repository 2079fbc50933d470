"""Pins of the oracle's EB geometry (Sec. "Embedded boundaries").

Checked against what geometry fixes on its own: exact volumes, apertures and
areas of planar cuts (inclusion-exclusion formulas for a half-space clipped
by a cube), and the O(h^2) convergence of the sphere's volume and area.
"""
import itertools

import numpy as np
import pytest


def _cut_volume(nv, d):
    """Volume of {x in [0,1]^3 : n.x < d} for n > 0 componentwise."""
    s = 0.0
    for v in itertools.product((0, 1), repeat=3):
        t = d - float(np.dot(nv, v))
        if t > 0:
            s += (-1) ** sum(v) * t ** 3
    return s / (6.0 * nv[0] * nv[1] * nv[2])


def _cut_area(nv, d):
    """Area of the plane n.x = d inside [0,1]^3, |n| = 1, n > 0."""
    s = 0.0
    for v in itertools.product((0, 1), repeat=3):
        t = d - float(np.dot(nv, v))
        if t > 0:
            s += (-1) ** sum(v) * t ** 2
    return s / (2.0 * nv[0] * nv[1] * nv[2])


def _cut_square(a, b, c):
    """Area of {(s,t) in [0,1]^2 : a s + b t < c}, a, b > 0."""
    s = 0.0
    for v in itertools.product((0, 1), repeat=2):
        t = c - a * v[0] - b * v[1]
        if t > 0:
            s += (-1) ** sum(v) * t ** 2
    return s / (2.0 * a * b)


@pytest.fixture(scope="module")
def plane_case(O):
    nv = np.array([1.0, 2.0, 3.0])
    nv /= np.linalg.norm(nv)
    d = 0.93
    n = 12
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_PLANE, p=tuple(nv) + (d,)))
    return g, geo, nv, d


def test_plane_volume_fraction_exact(O, plane_case):
    g, geo, nv, d = plane_case
    h, n = g.h, g.n[0]
    a = geo.alpha.reshape(g.cshape())
    for k, j, i in itertools.product(range(n), repeat=3):
        lo = np.array([i, j, k]) * h
        dl = (d - float(np.dot(nv, lo))) / h
        exact = 1.0 - min(max(_cut_volume(nv, dl), 0.0), 1.0)
        assert abs(a[k, j, i] - exact) < 1e-11, (i, j, k, a[k, j, i], exact)


def test_plane_apertures_exact(O, plane_case):
    g, geo, nv, d = plane_case
    h, n = g.h, g.n[0]
    ax = geo.ax.reshape(g.fshape(0))
    az = geo.az.reshape(g.fshape(2))
    for k, j, i in itertools.product(range(n), range(n), range(n + 1)):
        # x-face at x = i h spanning (y, z) cell (j, k): fluid where n.x > d
        c = (d - nv[0] * i * h - nv[1] * j * h - nv[2] * k * h) / h
        exact = 1.0 - min(max(_cut_square(nv[1], nv[2], c), 0.0), 1.0)
        assert abs(ax[k, j, i] - exact) < 1e-11
    for k, j, i in itertools.product(range(n + 1), range(n), range(n)):
        c = (d - nv[0] * i * h - nv[1] * j * h - nv[2] * k * h) / h
        exact = 1.0 - min(max(_cut_square(nv[0], nv[1], c), 0.0), 1.0)
        assert abs(az[k, j, i] - exact) < 1e-11


def test_plane_normal_area_centroid(O, plane_case):
    g, geo, nv, d = plane_case
    h, n = g.h, g.n[0]
    N3 = g.ncell
    cut = np.nonzero(geo.flag == 2)[0]
    assert len(cut) > 50
    nrm = geo.nrm.reshape(3, N3)[:, cut]
    b = geo.bcen.reshape(3, N3)[:, cut]
    # every cut cell sees the plane's own unit normal, pointing into the fluid
    assert np.abs(nrm - nv[:, None]).max() < 1e-12
    k, j, i = np.unravel_index(cut, g.cshape())
    centre = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h])
    # the EB centroid lies on the plane
    assert np.abs(nv @ (centre + h * b) - d).max() < 1e-12
    for q, c in enumerate(cut):
        lo = np.array([i[q], j[q], k[q]]) * h
        dl = (d - float(np.dot(nv, lo))) / h
        assert abs(geo.area[c] - _cut_area(nv, dl)) < 1e-11


@pytest.mark.parametrize("r", [0.125, 0.2])
def test_sphere_volume_area_second_order(O, r):
    errs_v, errs_a = [], []
    for n in (16, 32, 64):
        g = O.Grid(n=(n, n, n), h=1.0 / n)
        geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, r)))
        h = g.h
        errs_v.append(abs(geo.alpha.sum() * h ** 3 - (1 - 4.0 / 3.0 * np.pi * r ** 3)))
        errs_a.append(abs(geo.area.sum() * h ** 2 - 4 * np.pi * r ** 2))
        # normals point away from the sphere centre (into the fluid)
        cut = np.nonzero(geo.flag == 2)[0]
        k, j, i = np.unravel_index(cut, g.cshape())
        cen = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h]) - 0.5
        nrm = geo.nrm.reshape(3, -1)[:, cut]
        assert (np.sum(cen * nrm, axis=0) > 0).all()
    rv = np.log2(errs_v[1] / errs_v[2])
    ra = np.log2(errs_a[1] / errs_a[2])
    assert rv > 1.8 and ra > 1.8, (errs_v, errs_a)


def test_closure_and_flags(O):
    g = O.Grid(n=(16, 16, 16), h=1.0 / 16)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.27)))
    a = geo.alpha
    assert set(np.unique(geo.flag)) <= {0, 1, 2}
    assert (a[geo.flag == 0] == 0).all() and (a[geo.flag == 1] == 1).all()
    assert ((a[geo.flag == 2] > 0) & (a[geo.flag == 2] <= 1)).all()
    # area vector = difference of opposite apertures (closed fluid region)
    ax = geo.ax.reshape(g.fshape(0))
    ay = geo.ay.reshape(g.fshape(1))
    az = geo.az.reshape(g.fshape(2))
    An = np.stack([ax[:, :, 1:] - ax[:, :, :-1], ay[:, 1:, :] - ay[:, :-1, :],
                   az[1:, :, :] - az[:-1, :, :]]).reshape(3, -1)
    cut = geo.flag == 2
    An_eb = geo.nrm.reshape(3, -1) * geo.area
    assert np.abs(An[:, cut] - An_eb[:, cut]).max() < 1e-12

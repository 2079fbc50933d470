"""Pins of the oracle's flow diagnostics (Sec. "Cylinder moving through
Bingham fluid"): the flow topology parameter of Eq. ryovar,
Lambda = (||g||^2 - |w|^2) / (||g||^2 + |w|^2), is -1 for a rigid rotation,
0 for simple shear and 1 for pure extension, and for any linear field equals
the value computed from its constant velocity-gradient matrix; the relative
deviation from the yield stress, eta ||g|| / tau0 - 1, vanishes at the
regularised yield strain eps W(Bi/eps) and has the sign of ||g|| - that
strain.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _box(O, n=12):
    g = O.Grid(n=(n, n + 2, n + 4), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    nz, ny, nx = g.cshape()
    z, y, x = np.meshgrid(*[(np.arange(m) + 0.5) * g.h for m in (nz, ny, nx)], indexing="ij")
    return g, geo, x, y, z


def _linear_u(A, x, y, z):
    X = np.stack([x, y, z])
    return np.concatenate([np.tensordot(A[q], X, axes=1).ravel() for q in range(3)])


def _lambda_of(A):
    # A[q, d] = du_q / dx_d
    S = A + A.T
    s2 = 0.5 * (S * S).sum()
    w = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    w2 = (w * w).sum()
    return (s2 - w2) / (s2 + w2)


@pytest.mark.parametrize("A,expect", [
    (np.array([[0.0, -0.7, 0.0], [0.7, 0.0, 0.0], [0.0, 0.0, 0.0]]), -1.0),   # rotation about z
    (np.array([[0.0, 0.0, 1.3], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), 0.0),     # u = (g z, 0, 0)
    (np.array([[0.4, 0.0, 0.0], [0.0, -0.4, 0.0], [0.0, 0.0, 0.0]]), 1.0),    # planar extension
    (np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.25, 0.2, -0.7]]), None),
])
def test_lambda_of_linear_fields(O, A, expect):
    g, geo, x, y, z = _box(O)
    P = O.Params(mu=1.0, tau0=0.0, model=O.NEWTONIAN)
    lam, _ = O.flow_diagnostics(g, geo, P, _linear_u(A, x, y, z))
    ref = _lambda_of(A) if expect is None else expect
    if expect is not None:
        assert _lambda_of(A) == pytest.approx(expect, abs=1e-15)
    assert np.abs(lam - ref).max() < 1e-12


def test_stress_deviation_at_the_yield_strain(O):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "yield_strain.txt"))
            if l.strip() and not l.startswith("#")]
    bi, eps, printed = map(float, rows[0])
    g, geo, x, y, z = _box(O)
    P = O.Params(mu=1.0, tau0=bi, m=1.0 / eps, model=O.BINGHAM)
    # simple shear u = (s z, 0, 0) has ||g|| = s: the deviation crosses 0 at the printed strain
    for s, sign in ((printed, 0), (0.5 * printed, -1), (2.0 * printed, 1)):
        A = np.zeros((3, 3))
        A[0, 2] = s
        _, dev = O.flow_diagnostics(g, geo, P, _linear_u(A, x, y, z))
        expect = O.eta_of(P, s) * s / bi - 1.0
        assert np.abs(dev - expect).max() < 1e-12
        if sign == 0:
            assert abs(expect) < 2e-4   # the printed strain carries 5 digits
        else:
            assert np.sign(expect) == sign

"""Spatio-temporal convergence of the whole step (Sec. "Spatio-temporal
convergence study: Taylor-Green vortices", Eq. taylor-green, Table
tab:convergence): the Taylor-Green vortex at Re = 100 in the unit square
(8 cells deep, n/8 from 128^2), slip walls on all sides (the paper's
periodic solution also satisfies them exactly), advanced to t = 0.25 with
the step of Eqs. cfl:dt .. cfl:viscous:new (the last step shortened to end
there) on 64^2, 128^2 and 256^2 cells.  The velocity error at the cell
centres against the exact solution must fall at second order (rate > 1.8)
from 128^2 to 256^2 in the discrete L1, L2 and max norms, and by more than
1.4 from 64^2 to 128^2; the paper's rates also approach 2 only on the finer
grids, and its values are not targets (domain, end time and walls differ).
Algorithm 1 applies the implicit viscous operator with the full step in both
stages, which is first order in time for that part; the CFL step's viscous
limit makes the step O(h^2) on fine grids, so the run as a whole converges at
second order, as in the paper.  Also the first steps against the oracle, on a
box with no outflow side (both pressure problems fixed by the one reference
point).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
RE, T = 100.0, 0.25


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


def _solver(E, n, precision, tol):
    from paper_1905_07392_gb300 import workloads as W
    shape, h = W.taylor_green_grid(n)
    s = E.Solver(shape, h, bc=W.TG_BC, u_in=(0.0, 0.0, 0.0), rho=1.0, mu=1.0 / RE, tau0=0.0,
                 model=E.NEWTONIAN, tol=tol, max_iters=5000, precision=precision)
    s.build_geometry(lambda x: 1.0)
    return s


def _errors(E, n, precision):
    from paper_1905_07392_gb300 import workloads as W
    s = _solver(E, n, precision, 1e-12)
    u = torch.tensor(W.taylor_green_velocity(n).ravel(), device=DEV)
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    t = 0.0
    while t < T * (1.0 - 1e-12):
        dt = min(s.timestep(u), T - t)
        s.advance(u, p, dt=dt, stats=False)
        t += dt
    ue = W.taylor_green_velocity(n, t=T, re=RE)
    e = u.cpu().numpy().reshape(ue.shape) - ue
    mag = np.sqrt((e * e).sum(axis=0))
    s.close()
    return mag.mean(), np.sqrt((mag * mag).mean()), mag.max()


@pytest.mark.parametrize("precision", [0, 1])
def test_taylor_green_second_order(E, precision):
    errs = [_errors(E, n, precision) for n in (64, 128, 256)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates[-1] > 1.8).all(), (errs, rates)
    assert (rates[0] > 1.4).all(), (errs, rates)
    assert errs[-1][2] < 1e-4, errs


def test_taylor_green_steps_match_oracle(E, O):
    from paper_1905_07392_gb300 import workloads as W
    n = 16
    shape, h = W.taylor_green_grid(n)
    g = O.Grid(n=shape, h=h, bc=W.TG_BC, u_in=(0.0, 0.0, 0.0))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_NONE))
    P = O.Params(rho=1.0, mu=1.0 / RE, tau0=0.0, model=O.NEWTONIAN, tol=1e-13)
    s = _solver(E, n, 0, 1e-13)
    u0 = W.taylor_green_velocity(n).ravel()
    uo, po = u0.copy(), np.zeros(g.nnode)
    u = torch.tensor(u0, device=DEV)
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    for _ in range(3):
        uo, po, sto = O.advance(g, geo, P, uo, po, dt=0.25 / n)
        st = s.advance(u, p, dt=0.25 / n)
        ug = u.cpu().numpy()
        assert np.linalg.norm(ug - uo) <= 1e-10 * np.linalg.norm(uo)
        assert np.linalg.norm(p.cpu().numpy() - po) <= 1e-10 * np.linalg.norm(po)
    # the reference point of the nodal pressure
    assert po[0] == 0.0 and float(p[0]) == 0.0

"""The captured step (ebv_advance_graph): one CUDA graph per step whose solver
loops are conditional WHILE nodes.  It issues the same kernels with the same
arguments in the same order as the eager step, so the two agree bit for bit,
and it agrees with the FP64 oracle to the parity bar (1e-10 relative L2)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


def _solver(E, n, precision, tol=1e-12, **kw):
    s = E.Solver((n, n, n), 1.0 / n, tol=tol, max_iters=5000, precision=precision, tau0=1.0, m=1e3,
                 bi_cfl=0.25, **kw)
    s.build_sphere((0.5, 0.5, 0.5), 0.125)
    return s


def _state(s, n, seed):
    alpha = s.geometry()["alpha"].cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-1e-3, 1e-3, size=(3, n ** 3))
    u[2] += 1.0
    u = (u * (alpha > 0)).ravel()
    return (torch.tensor(u, device=DEV), torch.zeros((n + 1) ** 3, dtype=torch.float64, device=DEV))


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_steps_match_eager_bitwise(E, precision):
    n = 32
    s = _solver(E, n, precision)
    u1, p1 = _state(s, n, 3)
    u2, p2 = u1.clone(), p1.clone()
    l0 = s.launch_count()
    for i in range(3):
        st_e = s.advance(u1, p1, stats=(i == 2))
    l1 = s.launch_count()
    st_g = s.advance_graph(u2, p2, steps=3)
    l2 = s.launch_count()
    assert torch.equal(u1, u2) and torch.equal(p1, p2)
    assert st_g["iters"] == st_e["iters"]
    assert st_g["res"] == st_e["res"]
    assert st_g["dt"] == st_e["dt"] and st_g["drag"] == st_e["drag"]
    # launch accounting of the graph (captured body sizes x device iteration
    # counts) equals the eager count of the same three steps
    assert l2 - l1 == l1 - l0


def test_graph_matches_oracle(E, O):
    n = 32
    bc = (O.SLIP, O.SLIP, O.SLIP, O.SLIP, O.INFLOW, O.OUTFLOW)
    s = E.Solver((n, n, n), 1.0 / n, tol=1e-13, max_iters=5000, precision=1, tau0=1.0, m=1e3,
                 bi_cfl=0.25)
    s.build_sphere((0.5, 0.5, 0.5), 0.125)
    g = O.Grid(n=(n, n, n), h=1.0 / n, bc=bc, u_in=(0, 0, 1))
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=(0.5, 0.5, 0.5, 0.125)))
    P = O.Params(rho=1.0, mu=1.0, tau0=1.0, m=1e3, model=O.BINGHAM, bi_cfl=0.25, tol=1e-13,
                 max_iters=200000)
    rng = np.random.Generator(np.random.PCG64(21))
    u0 = rng.uniform(-1e-3, 1e-3, size=(3, g.ncell))
    u0[2] += 1.0
    u0 = (u0 * (geo.alpha > 0)).ravel()
    uo, po = u0.copy(), np.zeros(g.nnode)
    for _ in range(2):
        uo, po, sto = O.advance(g, geo, P, uo, po)
    u = torch.tensor(u0, device=DEV)
    p = torch.zeros(g.nnode, dtype=torch.float64, device=DEV)
    st = s.advance_graph(u, p, steps=2)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert max(st["res"]) <= 1e-13
    assert rel(u.cpu().numpy(), uo) < 1e-10
    assert rel(p.cpu().numpy(), po) < 1e-10
    assert st["drag"] == pytest.approx(sto["drag"], rel=1e-9)


def test_graph_recaptures_for_new_buffers(E):
    n = 16
    s = _solver(E, n, 1)
    ua, pa = _state(s, n, 5)
    ub, pb = _state(s, n, 6)
    ra, qa = ua.clone(), pa.clone()
    rb, qb = ub.clone(), pb.clone()
    s.advance_graph(ua, pa, steps=2, stats=False)
    s.advance_graph(ub, pb, steps=2, stats=False)
    s.advance_graph(ua, pa, steps=1, stats=False)
    for _ in range(3):
        s.advance(ra, qa, stats=False)
    for _ in range(2):
        s.advance(rb, qb, stats=False)
    assert torch.equal(ua, ra) and torch.equal(pa, qa)
    assert torch.equal(ub, rb) and torch.equal(pb, qb)


def test_graph_reports_failed_solve_and_recovers(E):
    n = 16
    s = _solver(E, n, 0)
    u, p = _state(s, n, 7)
    s.set_params(max_iters=1, tol=1e-15)
    with pytest.raises(E.EbvError) as ei:
        s.advance_graph(u, p, steps=1)
    assert ei.value.status == -3
    assert "slot" in str(ei.value)
    s.set_params(max_iters=5000, tol=1e-12)
    u, p = _state(s, n, 7)
    st = s.advance_graph(u, p, steps=1)
    assert max(st["res"]) <= 1e-12

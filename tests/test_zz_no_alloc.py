"""ebv_drag_noalloc: the drag and unyielded fraction for callers that cannot
allocate GPU memory (a memory pool they do not own, no device-memory growth
after start-up, or only the buffers they are handed).  It must give what
ebv_drag gives, on consecutive calls that share its fixed working storage.

Kept in a file collected last, so that a failing run stops after every other
test has run.
"""
import ctypes as C

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


def _state(E, W, w, steps=2):
    s = E.Solver.from_workload(w, tol=1e-10)
    geo = s.geometry()
    alpha = geo["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device="cuda") * (alpha > 0))
    u = u.reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        s.advance(u, p, stats=False)
    cut = torch.nonzero(geo["flag"] == 2).flatten().to(torch.int32).contiguous()
    assert cut.numel() > 0
    return s, geo, cut, u, p


def _check(E, s, geo, cut, u, p, stream=None):
    fz, yf = s.drag(u, p)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    E.drag_noalloc(s, geo, cut, u, p, out, stream=stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(fz, rel=1e-12), (got, fz)
    assert got[1] == pytest.approx(yf, abs=1e-12), (got, yf)


def test_noalloc_drag_matches_drag_on_consecutive_calls(E):
    from paper_1905_07392_gb300 import workloads as W
    # first the largest accepted grid (64^3 = 262,144 cells, the inclusive
    # limit), then a smaller one, so the second call runs over storage the
    # first one filled with a different grid and cut list
    w64 = W.sphere_channel_32()
    w64.n = 64
    s64, geo64, cut64, u64, p64 = _state(E, W, w64, steps=1)
    _check(E, s64, geo64, cut64, u64, p64)
    w = W.sphere_channel_32()
    s, geo, cut, u, p = _state(E, W, w)
    assert cut.numel() < cut64.numel()
    for uu, pp in [(u, p), (u * 0.5, p + 3.0)]:  # the second call sees a different state
        _check(E, s, geo, cut, uu, pp)
    # a call queued on a stream of its own
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        _check(E, s, geo, cut, u, p, stream=side)
    # and the large grid again after the small one
    _check(E, s64, geo64, cut64, u64, p64)
    # sizes beyond the fixed storage are refused before any GPU work
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    g = E._Grid()
    g.n[:] = [128, 128, 128]
    g.h = 1.0 / 128
    dummy = C.c_void_p(out.data_ptr())
    st = E.load().ebv_drag_noalloc(C.byref(g), C.byref(s._params_c()), dummy, dummy, dummy, dummy,
                                   dummy, dummy, C.c_int(1), dummy, dummy, dummy, None)
    assert st == -7
    # h <= 0 is refused
    g.n[:] = [32, 32, 32]
    g.h = 0.0
    st = E.load().ebv_drag_noalloc(C.byref(g), C.byref(s._params_c()), dummy, dummy, dummy, dummy,
                                   dummy, dummy, C.c_int(1), dummy, dummy, dummy, None)
    assert st == -1

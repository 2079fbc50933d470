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


def test_noalloc_drag_matches_drag_on_consecutive_calls(E):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    s = E.Solver.from_workload(w, tol=1e-10)
    geo = s.geometry()
    alpha = geo["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device="cuda") * (alpha > 0))
    u = u.reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.advance(u, p, stats=False)
    cut = torch.nonzero(geo["flag"] == 2).flatten().to(torch.int32).contiguous()
    assert cut.numel() > 0
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    states = [(u, p), (u * 0.5, p + 3.0)]  # the second call sees a different state
    for uu, pp in states:
        fz, yf = s.drag(uu, pp)
        out.fill_(float("nan"))
        E.drag_noalloc(s, geo, cut, uu, pp, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(fz, rel=1e-12), (got, fz)
        assert got[1] == pytest.approx(yf, abs=1e-12), (got, yf)
    # sizes beyond the fixed storage are refused before any GPU work
    g = E._Grid()
    g.n[:] = [128, 128, 128]
    g.h = 1.0 / 128
    dummy = C.c_void_p(out.data_ptr())
    st = E.load().ebv_drag_noalloc(C.byref(g), C.byref(s._params_c()), dummy, dummy, dummy, dummy,
                                   dummy, dummy, C.c_int(1), dummy, dummy, dummy, None)
    assert st == -7

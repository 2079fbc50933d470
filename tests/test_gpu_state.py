"""Checkpoint and restart (ebv_save_state / ebv_load_state): a run saved
after some steps and resumed in a fresh context, created with other
parameters and no geometry, continues bit for bit as the uninterrupted run;
the loaded geometry equals the saved one bit for bit; a file saved on another
grid, or a file that is not a state, is refused."""
import os

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


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_is_bitwise(E, tmp_path, precision):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_32()
    s = E.Solver.from_workload(w, precision=precision, tol=1e-10, max_iters=2000)
    alpha = s.geometry()["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=DEV) * (alpha > 0)).reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    for _ in range(2):
        s.advance(u, p, stats=False)
    path = str(tmp_path / "state.ebv")
    s.save_state(u, p, path)
    for _ in range(3):
        s.advance(u, p, stats=False)
    # a fresh context on the same grid, other parameters, no geometry
    r = E.Solver((w.n,) * 3, w.h, tau0=7.0, m=10.0, tol=1e-6, precision=1 - precision)
    u2 = torch.full_like(u, float("nan"))
    p2 = torch.full_like(p, float("nan"))
    r.load_state(u2, p2, path)
    g1, g2 = s.geometry(), r.geometry()
    for k in g1:
        assert torch.equal(g1[k], g2[k]), k
    for _ in range(3):
        r.advance(u2, p2, stats=False)
    assert torch.equal(u, u2) and torch.equal(p, p2)
    # another grid, or not a state file
    q = E.Solver((16, 16, 16), 1.0 / 16, tol=1e-8)
    with pytest.raises(E.EbvError) as ei:
        q.load_state(torch.zeros(3 * 16 ** 3, dtype=torch.float64, device=DEV),
                     torch.zeros(17 ** 3, dtype=torch.float64, device=DEV), path)
    assert ei.value.status == -1
    bad = tmp_path / "bad.ebv"
    bad.write_bytes(b"not a state file at all")
    with pytest.raises(E.EbvError):
        r.load_state(u2, p2, str(bad))
    for x in (s, r, q):
        x.close()

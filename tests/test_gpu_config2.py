"""The 128^3 sphere-channel configuration against the oracle: Bingham numbers
0, 1 and 10 (tau0 = Bi mu U / (2 r)) and Herschel-Bulkley n = 0.5, r = 0.125,
m = 1e3, two CFL steps from the seeded noisy inflow, every solve to 1e-13,
in both precisions.

The oracle's results come from tests/golden/config2_sphere_channel_128.json,
written by tests/golden/make_config2.py, which calls only the oracle (a
128^3 oracle step takes minutes).  Compared per step: the time step (1e-12),
drag (Eq. drag-force, 1e-9) and the Stokes coefficient C_S = F_D/(6 pi mu U R)
(Eq. drag-coef), and the unyielded fraction (to 1e-6: one cell's eta s sitting
on the (1 + 1e-3) tau0 threshold moves it by about 5e-7); after the last step
the 2-norms of u and p (1e-10) and u, p at 512 seeded cells and nodes (1e-10
of the field's largest sampled magnitude).
"""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config2_sphere_channel_128.json")


def _cases():
    if not os.path.exists(GOLDEN):
        return []
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    return ebvisc


def _workload(name):
    from paper_1905_07392_gb300 import workloads as W
    if name == "hb_n0.5":
        return W.sphere_channel_128(herschel_bulkley=True)
    return W.sphere_channel_128(float(name[2:]))


def test_golden_file_present():
    assert len(_cases()) == 4


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("ref", _cases(), ids=lambda r: r["case"])
def test_config2_against_oracle(E, ref, precision):
    from paper_1905_07392_gb300 import workloads as W
    w = _workload(ref["case"])
    assert (w.n, w.tau0, w.n_flow, w.model) == (ref["n"], ref["tau0"], ref["n_flow"], ref["model"])
    s = E.Solver.from_workload(w, precision=precision, tol=ref["tol"], max_iters=20000)
    alpha = s.geometry()["alpha"]
    u = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=DEV) * (alpha > 0)).reshape(-1).contiguous()
    p = torch.zeros(s.nnode, dtype=torch.float64, device=DEV)
    for k in range(ref["steps"]):
        st = s.advance(u, p)
        assert max(st["res"]) <= ref["tol"]
        assert st["dt"] == pytest.approx(ref["dt"][k], rel=1e-12)
        assert st["drag"] == pytest.approx(ref["drag"][k], rel=1e-9)
        c_s = st["drag"] / (6.0 * math.pi * w.mu * 1.0 * w.radius)
        assert c_s == pytest.approx(ref["c_s"][k], rel=1e-9)
        assert st["yield_frac"] == pytest.approx(ref["yield_frac"][k], abs=1e-6)
    assert float(torch.linalg.vector_norm(u)) == pytest.approx(ref["u_norm"], rel=1e-10)
    assert float(torch.linalg.vector_norm(p)) == pytest.approx(ref["p_norm"], rel=1e-10)
    U = u.reshape(3, -1)[:, torch.tensor(ref["cells"], device=DEV)].T.cpu().numpy()
    Uo = np.array(ref["u"])
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()
    P = p[torch.tensor(ref["nodes"], device=DEV)].cpu().numpy()
    Po = np.array(ref["p"])
    assert np.abs(P - Po).max() <= 1e-10 * np.abs(Po).max()

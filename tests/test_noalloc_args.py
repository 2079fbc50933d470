"""Argument checks of the binding of ebv_drag_noalloc (host only, no GPU).

The C entry receives bare pointers and cannot see buffer sizes, so the binding
refuses every short, long or mistyped buffer, and cut lists with entries
outside the grid, before anything reaches the library.
"""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1905_07392_gb300 import ebvisc as E  # noqa: E402


def _case(n=4):
    g = E._Grid()
    g.n[:] = [n, n, n]
    g.h = 1.0 / n
    n3, nn = n ** 3, (n + 1) ** 3
    geo = {"alpha": torch.ones(n3, dtype=torch.float64), "area": torch.zeros(n3, dtype=torch.float64),
           "nrm": torch.zeros(3 * n3, dtype=torch.float64), "bcen": torch.zeros(3 * n3, dtype=torch.float64),
           "flag": torch.ones(n3, dtype=torch.uint8)}
    cut = torch.tensor([1, 5], dtype=torch.int32)
    u = torch.zeros(3 * n3, dtype=torch.float64)
    p = torch.zeros(nn, dtype=torch.float64)
    out = torch.zeros(2, dtype=torch.float64)
    return g, geo, cut, u, p, out


def test_valid_arguments_pass_the_checks():
    E._check_noalloc_args(*_case())


@pytest.mark.parametrize("what", ["out_short", "out_f32", "u_short", "p_long", "alpha_short", "nrm_short",
                                  "bcen_f32", "flag_f64", "cut_i64", "cut_neg", "cut_big", "cut_long"])
def test_bad_arguments_are_refused(what):
    g, geo, cut, u, p, out = _case()
    n3 = 64
    if what == "out_short":
        out = torch.zeros(1, dtype=torch.float64)
    elif what == "out_f32":
        out = torch.zeros(2, dtype=torch.float32)
    elif what == "u_short":
        u = torch.zeros(3 * n3 - 1, dtype=torch.float64)
    elif what == "p_long":
        p = torch.zeros(126, dtype=torch.float64)
    elif what == "alpha_short":
        geo["alpha"] = torch.ones(n3 - 1, dtype=torch.float64)
    elif what == "nrm_short":
        geo["nrm"] = torch.zeros(n3, dtype=torch.float64)
    elif what == "bcen_f32":
        geo["bcen"] = torch.zeros(3 * n3, dtype=torch.float32)
    elif what == "flag_f64":
        geo["flag"] = torch.ones(n3, dtype=torch.float64)
    elif what == "cut_i64":
        cut = cut.to(torch.int64)
    elif what == "cut_neg":
        cut = torch.tensor([-1, 3], dtype=torch.int32)
    elif what == "cut_big":
        cut = torch.tensor([3, n3], dtype=torch.int32)
    elif what == "cut_long":
        cut = torch.arange(n3 + 1, dtype=torch.int32) % n3
    with pytest.raises(ValueError):
        E._check_noalloc_args(g, geo, cut, u, p, out)
    solver = types.SimpleNamespace(_grid=g, _params_c=E._Params)
    with pytest.raises(ValueError):  # refused before the library is reached
        E.drag_noalloc(solver, geo, cut, u, p, out)

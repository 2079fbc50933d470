"""Writes config2_sphere_channel_128.json: the oracle's results for the 128^3
sphere-channel cases (r = 0.125, m = 1e3; Bingham numbers 0, 1, 10 with
tau0 = Bi mu U / (2 r), and Herschel-Bulkley n = 0.5, tau0 = 1), each run for
STEPS steps of Algorithm 1 at the CFL time step from the seeded noisy inflow,
every linear solve to a relative residual of 1e-13.

Stored per case: the time step, drag (Eq. drag-force), Stokes drag
coefficient C_S = F_D / (6 pi mu U R) (Eq. drag-coef; mu is kappa for HB) and
unyielded fraction after each step; the 2-norms and sums of the final u and
p; and u (three components) at SAMPLES seeded cells and p at SAMPLES seeded
nodes.  Only the oracle and the seeded input module are called, so every
value here is the oracle's.  Run: python tests/golden/make_config2.py
(about 20 minutes on 8 cores).
"""
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1905_07392_gb300 import workloads as W  # noqa: E402

STEPS = 2
SAMPLES = 512
TOL = 1e-13
OUT = os.path.join(HERE, "config2_sphere_channel_128.json")


def cases():
    return [("bi0", W.sphere_channel_128(0.0)), ("bi1", W.sphere_channel_128(1.0)),
            ("bi10", W.sphere_channel_128(10.0)), ("hb_n0.5", W.sphere_channel_128(herschel_bulkley=True))]


def sample_indices(ncell, nnode):
    rng = np.random.Generator(np.random.PCG64(2024))
    return (np.sort(rng.choice(ncell, SAMPLES, replace=False)),
            np.sort(rng.choice(nnode, SAMPLES, replace=False)))


def run_case(name, w):
    n = w.n
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (w.radius,)))
    P = O.Params(rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m, n_flow=w.n_flow, model=w.model, cfl=w.cfl,
                 bi_cfl=w.bingham, tol=TOL)
    u = (W.initial_velocity(w).reshape(3, -1) * (geo.alpha > 0)).ravel()
    p = np.zeros(g.nnode)
    rec = {"case": name, "n": n, "radius": w.radius, "tau0": w.tau0, "m": w.m, "n_flow": w.n_flow,
           "model": w.model, "bingham": w.bingham, "tol": TOL, "steps": STEPS,
           "dt": [], "drag": [], "c_s": [], "yield_frac": [], "iters": []}
    for _ in range(STEPS):
        u, p, st = O.advance(g, geo, P, u, p)
        rec["dt"].append(st["dt"])
        rec["drag"].append(st["drag"])
        rec["c_s"].append(st["drag"] / (6.0 * math.pi * w.mu * 1.0 * w.radius))
        rec["yield_frac"].append(st["yield_frac"])
        rec["iters"].append(st["iters"])
    cells, nodes = sample_indices(g.ncell, g.nnode)
    U = u.reshape(3, -1)
    rec.update({"u_norm": float(np.linalg.norm(u)), "p_norm": float(np.linalg.norm(p)),
                "u_sum": float(u.sum()), "p_sum": float(p.sum()),
                "cells": cells.tolist(), "u": U[:, cells].T.tolist(),
                "nodes": nodes.tolist(), "p": p[nodes].tolist()})
    return rec


def main():
    out = {"generator": "tests/golden/make_config2.py", "source": "oracle/ (FP64, OpenMP)", "cases": []}
    for name, w in cases():
        t0 = time.time()
        out["cases"].append(run_case(name, w))
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()

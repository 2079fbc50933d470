"""Throughput of the embedded-boundary viscoplastic step on GB300.

Workload: sphere-in-channel on [0,1]^3 at 256^3 cells, sphere r = 0.1 at the
centre, Bi = 10 (tau0 = 50), Papanastasiou m = 1e4, inflow (0,0,1) at z = 0,
outflow at z = 1, slip walls; seeded uniform noise of amplitude 1e-3 on the
inflow value (synthetic; the paper's sphere study is the template).  A step is
one full two-stage Runge-Kutta step (Algorithm 1): derived quantities, six
viscous solves, two cell-centred and two nodal projections, solved to a
relative residual of 1e-8.  The metric is Mcell-steps/s = cells * steps /
seconds / 1e6 for the FP32-smoother / FP64-refinement path; the FP64 path is
measured in the same run.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank advances its own replica (the problem does
not shard: one problem's solves would need a halo exchange per smoother pass
and an all-reduce per dot product) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s at 256^3 (FP32+refine, 1e-8 tol)"
UNIT = "Mcell-steps/s"
CPU_SAMPLE_N = 64  # oracle sample grid (same problem, coarser grid)
PRECISION = ("FP64 iterative refinement (FP64 operator, residual and solution) around FP32 conjugate "
             "gradients preconditioned by an FP32 multigrid V-cycle whose cell-centred face coefficients "
             "are stored in BF16 (nodal V-cycle FP32); geometry and fields FP64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per side (256 is the workload)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-fp32-faces", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--skip-config2", action="store_true")
    ap.add_argument("--skip-paper", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=CPU_SAMPLE_N,
                    help="grid of the oracle sample (cpu_baseline and the reference arm)")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle on the 128^3 sphere channel (minutes)")
    ap.add_argument("--eager", action="store_true",
                    help="issue every step kernel by kernel (no step graph), e.g. under a profiler")
    ap.add_argument("--inner-drop", type=float, default=1e-4,
                    help="residual drop of each FP32 correction solve of the refinement (ebv_set_inner_drop)")
    ap.add_argument("--fused-sweep", type=int, default=1, choices=[0, 1, 2],
                    help="smoother sweeps of FP32 levels: 0 colour passes, 1 the faster form per level "
                         "(timed at set-up, default), 2 the fused one-pass sweep (same results)")
    return ap.parse_args()


def workload(n):
    from paper_1905_07392_gb300 import workloads as W
    w = W.sphere_channel_256()
    if n != 256:
        w.n = n
    return w


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_init(args):
    """Rank, world size and local rank from the launcher's environment; for
    world > 1 a process group over NCCL (one GPU per rank), or over gloo on a
    host without CUDA (the same plumbing, exercised by the CPU tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over all ranks (the timed region's slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells, steps, world, sec):
    """Whole-job Mcell-steps/s: every rank advances its own replica of `cells`
    cells for `steps` steps; sec is the slowest rank's time."""
    return cells * steps * world / sec / 1e6


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_solver(w, precision, tol=1e-8, lib=None):
    from paper_1905_07392_gb300 import ebvisc
    return ebvisc.Solver.from_workload(w, precision=precision, tol=tol, max_iters=2000, lib=lib)


def initial_state(s, w, dev):
    import numpy as np
    import torch
    from paper_1905_07392_gb300 import workloads as W
    alpha = s.geometry()["alpha"]
    u0 = torch.tensor(W.initial_velocity(w).reshape(3, -1), device=dev)
    u0 = (u0 * (alpha > 0)).reshape(-1).contiguous()
    p0 = torch.zeros(s.nnode, dtype=torch.float64, device=dev)
    return u0, p0


def time_steps(s, u, p, steps, warmup, world, profile=False, graph=False):
    """Warm-up, then exactly `steps` steps between barriers and syncs, timed
    with CUDA events on the solver's stream.  graph: each step is one launch
    of the captured step graph (captured during the warm-up); otherwise the
    step's kernels are issued one by one (with profile: each bracketed by
    CUDA events).  Returns (seconds, kernel launches, profile or None)."""
    import torch
    if graph:
        s.advance_graph(u, p, steps=warmup, stats=False)
    else:
        for _ in range(warmup):
            s.advance(u, p, stats=False)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = s.launch_count()
    if profile:
        s.profile_begin()
    e0.record(s.stream)
    if graph:
        s.advance_graph(u, p, steps=steps, stats=False)
    else:
        for _ in range(steps):
            s.advance(u, p, stats=False)
    e1.record(s.stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    prof = s.profile_end() if profile else None
    return sec, s.launch_count() - launches0, prof


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM bytes (read + write) per algorithmic byte, from one ncu capture of the
# current kernel on a smaller grid (192^3, traffic grows with the cells);
# the reported traffic is this ratio times the algorithmic bytes per launch.
# The fused sweep's figure is over its four kinds (from zero, plain, after the
# coarse correction, with r.z), which share the L0 label.
NCU_TRAFFIC_RATIO = {"cc_gs_colour_pass<float> L0": 1.16, "cc_rb_sweep<float> L0": 0.97}


def roofline(prof, cells):
    """Roofline of the kernel with the largest summed time among those whose
    algorithmic bytes are stated: bytes per launch over the average
    CUDA-event launch duration.  Also the top kernels by time."""
    peak, src = measured_peaks()
    ks = {k: v for k, v in prof.items() if v["launches"] > 0}
    total = sum(v["ms"] for v in ks.values())
    kernels = {}
    for k, f in sorted(ks.items(), key=lambda kv: -kv[1]["ms"])[:24]:
        e = {"launches": f["launches"], "ms": round(f["ms"], 3),
             "share": round(f["ms"] / total, 4)}
        if f["bytes"] > 0:
            e["GB/s"] = round(f["bytes"] / (f["ms"] * 1e-3) / 1e9, 1)
        kernels[k] = e
    stated = {k: v for k, v in ks.items() if v["bytes"] > 0}
    top = max(stated, key=lambda k: stated[k]["ms"])
    v = stated[top]
    avg_ms = v["ms"] / v["launches"]
    bytes_per_launch = v["bytes"] / v["launches"]
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": peak,
            "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": (round(NCU_TRAFFIC_RATIO[top] * bytes_per_launch, 1)
                        if top in NCU_TRAFFIC_RATIO else None),
            "algorithmic_bytes_per_launch": round(bytes_per_launch, 1),
            "avg_launch_ms": round(avg_ms, 5)}, kernels


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_1905_07392_gb300 import build_lib, ebvisc
    build_lib.build()
    ebvisc.load().ebv_set_fused_sweep(args.fused_sweep)
    ebvisc.load().ebv_set_inner_drop(args.inner_drop)
    dev = torch.device("cuda", local)
    w = workload(args.n)
    cells = w.n ** 3

    # FP32 smoother + FP64 refinement (headline): each step one launch of the
    # captured step graph
    s = make_solver(w, ebvisc.FP32_REFINE)
    u, p = initial_state(s, w, dev)
    clocks = Clocks(local)
    clocks.start()
    sec, launches, _ = time_steps(s, u, p, args.steps, args.warmup, world, graph=not args.eager)
    ck = clocks.stop()
    sec = max_over_ranks(sec, world)
    st = s.advance(u.clone(), p.clone(), stats=True)
    # kernel breakdown and roofline: the same steps issued kernel by kernel,
    # each launch bracketed by CUDA events (graph nodes cannot be timed singly)
    ue, pe = initial_state(s, w, dev)
    sec_e, _, prof = time_steps(s, ue, pe, args.steps, args.warmup, world, profile=True)
    sec_e = max_over_ranks(sec_e, world)
    del ue, pe
    value = job_value(cells, args.steps, world, sec)
    roof, kernels = roofline(prof, cells)
    # the timings that chose each MAC level's sweep form (fused, passes; ms
    # of four launches) for the kinds from zero, plain, corrected, with r.z
    sweeps = {}
    for lv in range(8):
        try:
            t = [s.sweep_timing(lv, k) for k in range(4)]
        except Exception:
            break
        if any(f < 1e29 for f, _ in t):
            sweeps[f"L{lv}"] = {n: [round(f, 4), round(q, 4)]
                                for n, (f, q) in zip(("zero", "plain", "corr", "dot"), t) if f < 1e29}

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sec / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16",
           "data": "synthetic (seeded noise on uniform inflow; no dataset)",
           "config": {"workload": f"sphere_channel_{w.n}^3_bi10_m1e4", "cells": cells,
                      "sphere_radius": w.radius, "bingham": w.bingham, "m": w.m, "tol": 1e-8,
                      "precision": PRECISION,
                      "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs larger than L2 (each cell field 134 MB at 256^3)"},
           "roofline": roof, "kernels": kernels, "sweep_forms_ms": sweeps,
           "step_launch": ("kernel by kernel" if args.eager else
                           "one CUDA graph launch per step (solver loops as conditional nodes)"),
           "eager": {"value": round(job_value(cells, args.steps, world, sec_e), 3), "unit": UNIT,
                     "ms_per_step": round(1e3 * sec_e / args.steps, 3),
                     "note": "kernel-by-kernel issue with per-launch CUDA events; roofline and "
                             "kernels are measured here"},
           "clocks": ck, "gpu_launches": launches,
           "solve_iters_last_step": st["iters"], "dt": st["dt"], "drag": st["drag"],
           "yield_frac": st["yield_frac"]}
    s.close()

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    ref64 = None   # (u, p, stats) of the FP64 path after the timed steps, for the other forms
    if not args.skip_fp64:
        s64 = make_solver(w, ebvisc.FP64)
        u64, p64 = initial_state(s64, w, dev)
        sec64, _, _ = time_steps(s64, u64, p64, args.steps, args.warmup, world, graph=True)
        sec64 = max_over_ranks(sec64, world)
        st64 = s64.advance(u64.clone(), p64.clone(), stats=True)
        out["fp64"] = {"value": round(job_value(cells, args.steps, world, sec64), 3), "unit": UNIT,
                       "ms_per_step": round(1e3 * sec64 / args.steps, 3),
                       "solve_iters_last_step": st64["iters"]}
        # error of the FP32-smoother path against FP64 after the same steps
        # from the same seeded state
        ref64 = (u64, p64, st64)
        out["fp32_vs_fp64"] = {"steps": args.warmup + args.steps, "u_rel_l2": rel(u, u64),
                               "p_rel_l2": rel(p, p64),
                               "drag_rel": abs(st["drag"] - st64["drag"]) / abs(st64["drag"])}
        s64.close()

    if not args.skip_fp32_faces:
        # the same path with the V-cycle reading FP32 instead of BF16 face
        # coefficients (a build variant of the library: only the face type differs)
        from paper_1905_07392_gb300 import build_lib
        vlib = ebvisc.load_variant(build_lib.VARIANT_LIB)
        sf = make_solver(w, ebvisc.FP32_REFINE, lib=vlib)
        uf, pf = initial_state(sf, w, dev)
        secf, _, _ = time_steps(sf, uf, pf, args.steps, args.warmup, world, graph=True)
        secf = max_over_ranks(secf, world)
        stf = sf.advance(uf.clone(), pf.clone(), stats=True)
        out["fp32_faces"] = {"value": round(job_value(cells, args.steps, world, secf), 3), "unit": UNIT,
                             "ms_per_step": round(1e3 * secf / args.steps, 3),
                             "solve_iters_last_step": stf["iters"],
                             "note": "same step with the FP32 V-cycle reading FP32 face coefficients "
                                     "(library build variant EBV_VCYCLE_FP32_FACES); headline uses BF16"}
        sf.close()
        del uf, pf

    if not args.skip_mixed:
        # FP32_MIXED: the same path with the strain rate and viscosity of the
        # cells away from the EB in FP32; its error against FP64 after the same
        # steps, and the strain-rate kernel's achieved bandwidth (eager profile)
        sm = make_solver(w, ebvisc.FP32_MIXED)
        um, pm = initial_state(sm, w, dev)
        secm, _, _ = time_steps(sm, um, pm, args.steps, args.warmup, world, graph=True)
        secm = max_over_ranks(secm, world)
        stm = sm.advance(um.clone(), pm.clone(), stats=True)
        ue, pe = initial_state(sm, w, dev)
        _, _, profm = time_steps(sm, ue, pe, 2, 1, world, profile=True)
        del ue, pe
        mix = {"value": round(job_value(cells, args.steps, world, secm), 3), "unit": UNIT,
               "ms_per_step": round(1e3 * secm / args.steps, 3), "solve_iters_last_step": stm["iters"]}
        k5 = profm.get("strain_rate_viscosity")
        if k5 and k5["launches"] > 0:
            gbs = k5["bytes"] / (k5["ms"] * 1e-3) / 1e9
            mix["strain_rate_viscosity"] = {"ms_per_launch": round(k5["ms"] / k5["launches"], 4),
                                            "GB/s": round(gbs, 1), "frac": round(gbs / measured_peaks()[0], 4)}
        if ref64 is not None:
            u64, p64, st64 = ref64
            mix["vs_fp64"] = {"steps": args.warmup + args.steps, "u_rel_l2": rel(um, u64), "p_rel_l2": rel(pm, p64),
                              "drag_rel": abs(stm["drag"] - st64["drag"]) / abs(st64["drag"])}
        mix["note"] = ("precision EBV_FP32_MIXED: as the headline, with the strain rate and apparent viscosity "
                       "of cells away from the EB formed in FP32 from FP64 velocity differences")
        out["fp32_mixed"] = mix
        sm.close()
        del um, pm

    if not args.skip_config2:
        out["config2"] = run_config2(dev)
    if not args.skip_paper:
        try:
            out["paper_workloads"] = run_paper_workloads(dev)
        except Exception as e:  # reported in the line; the rest of the measurement stands
            out["paper_workloads"] = {"error": str(e)}

    if not args.skip_e2e:
        # end to end through the C-ABI with host buffers: every step copies
        # u and p host->device, advances, and copies them back
        s = make_solver(w, ebvisc.FP32_REFINE)
        u, p = initial_state(s, w, dev)
        uh = torch.empty(u.numel(), dtype=torch.float64, pin_memory=True)
        ph = torch.empty(p.numel(), dtype=torch.float64, pin_memory=True)
        uh.copy_(u.cpu())
        ph.copy_(p.cpu())
        un, pn = uh.numpy(), ph.numpy()
        for _ in range(args.warmup):
            s.advance_host(un, pn, 1)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.advance_host(un, pn, 1)
        t1 = time.perf_counter()
        barrier(world)
        se = max_over_ranks(t1 - t0, world)
        nb = 8 * (u.numel() + p.numel())
        out["e2e"] = {"value": round(job_value(cells, args.steps, world, se), 3), "unit": UNIT,
                      "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}
        s.close()

    if not args.skip_batch:
        out["batch_sweep"] = run_batch(dev, world)
    if not args.skip_adjoint:
        for key, adv in (("adjoint", 0), ("adjoint_full_step", 1)):
            try:
                out[key] = run_adjoint(dev, advect=adv)
            except Exception as e:  # reported in the line; the rest of the measurement stands
                out[key] = {"error": str(e)}
    return out


def run_config2(dev, steps=20, tol=1e-10):
    """The 128^3 sphere channel (r = 0.125, m = 1e3) for Bi in {0, 1, 10} and
    Herschel-Bulkley n = 0.5, FP64 path, 20 CFL steps each: drag F_D (Eq.
    drag-force), Stokes coefficient C_S = F_D / (6 pi mu U R) (Eq. drag-coef;
    mu is kappa for HB) and unyielded fraction after the last step."""
    import math
    import torch
    from paper_1905_07392_gb300 import ebvisc
    from paper_1905_07392_gb300 import workloads as W
    out = {"steps": steps, "tol": tol, "precision": "fp64", "cases": {}}
    for name, w in (("bi0", W.sphere_channel_128(0.0)), ("bi1", W.sphere_channel_128(1.0)),
                    ("bi10", W.sphere_channel_128(10.0)), ("hb_n0.5", W.sphere_channel_128(herschel_bulkley=True))):
        s = ebvisc.Solver.from_workload(w, precision=ebvisc.FP64, tol=tol, max_iters=5000)
        u, p = initial_state(s, w, dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps - 1):
            s.advance(u, p, stats=False)
        st = s.advance(u, p, stats=True)
        torch.cuda.synchronize()
        out["cases"][name] = {"bingham": round(w.bingham, 6), "F_D": st["drag"],
                              "C_S": st["drag"] / (6.0 * math.pi * w.mu * 1.0 * w.radius),
                              "yield_frac": st["yield_frac"], "dt": st["dt"],
                              "seconds": round(time.perf_counter() - t0, 3)}
        s.close()
    return out


def faxen_cd(d_over_w):
    """Faxen's creeping drag per unit length on a cylinder in a channel
    (Appendix "Faxen's formula", Eq. faxen), as C_D = F_D / (mu U L)."""
    import math
    k = d_over_w
    return 4.0 * math.pi / (math.log(1.0 / k) - 0.9157 + 1.7244 * k ** 2 - 1.7302 * k ** 4 + 2.4056 * k ** 6
                            - 4.5913 * k ** 8)


def steady_creeping(s, u, p, dt_mult=100.0, max_steps=300, rtol=1e-7):
    """Creeping-flow steps (advect = 0) at dt_mult times the CFL step of the
    initial state until the drag changes by less than rtol; the viscous
    update is implicit, so the large step only speeds up the approach to the
    steady state, which is the same at any step size.  Returns (stats, steps,
    the last step's relative drag change): steps == max_steps with a change
    above rtol means the cap ended the run."""
    dt = s.timestep(u) * dt_mult
    prev, rel = None, float("nan")
    for k in range(max_steps):
        st = s.advance(u, p, dt=dt)
        if prev is not None:
            rel = abs(st["drag"] - prev) / abs(st["drag"])
            if rel <= rtol:
                return st, k + 1, rel
        prev = st["drag"]
    return st, max_steps, rel


def run_paper_workloads(dev, cells_per_d=16):
    """The paper's flow-past-body set-ups at a coarse resolution (16 cells per
    diameter; the paper uses 64), steady creeping flow, FP32 + refinement to
    1e-10: the cylinder slab [0,4D] x [0,D/2] x [0,6D] (Newtonian, against
    Faxen's formula; slip walls in y stand for the periodic sides, the flow
    being uniform along the axis), the sphere box [0,4D]^2 x [0,6D] (Newtonian
    and Bi = 10, C_S = F_D / (6 pi mu U R), unyielded fraction) and the
    sphere-and-cube body (Bi = 10), each with u = U e_z on every side."""
    import math
    import torch
    from paper_1905_07392_gb300 import ebvisc as E
    from paper_1905_07392_gb300 import workloads as W
    D, npd = 0.25, cells_per_d
    h = D / npd
    out = {"cells_per_d": npd, "precision": "fp32_refine", "tol": 1e-10}

    def make(n, bc, bodies, tau0=0.0, model=E.NEWTONIAN):
        s = E.Solver(n, h, bc=bc, u_in=(0.0, 0.0, 1.0), mu=1.0, tau0=tau0, m=1e3, model=model, tol=1e-10,
                     max_iters=5000, advect=0, precision=E.FP32_REFINE, bi_cfl=tau0 * D)
        s.build_bodies(bodies)
        alpha = s.geometry()["alpha"]
        u = torch.zeros(3 * s.ncell, dtype=torch.float64, device=dev)
        u[2 * s.ncell:] = (alpha > 0).to(torch.float64)
        p = torch.zeros(s.nnode, dtype=torch.float64, device=dev)
        return s, u, p

    t0 = time.perf_counter()
    n = (4 * npd, npd // 2, 6 * npd)
    s, u, p = make(n, (W.INFLOW, W.INFLOW, W.SLIP, W.SLIP, W.INFLOW, W.INFLOW),
                   [(E.BODY_CYLINDER, (1, 2 * D, 3 * D, D / 2))])
    st, k, rel = steady_creeping(s, u, p)
    cd = st["drag"] / (1.0 * 1.0 * n[1] * h)
    out["cylinder_newtonian"] = {"C_D": cd, "faxen_C_D": faxen_cd(0.25), "rel_diff": cd / faxen_cd(0.25) - 1.0,
                                 "steps": k, "last_rel_change": rel, "cells": n[0] * n[1] * n[2]}
    s.close()
    n, hh = W.sphere_box_grid(npd, D)
    for bi in (0.0, 10.0):
        tau0 = W.tau0_for_bingham(bi, D / 2)
        s, u, p = make(n, (W.INFLOW,) * 6, [(E.BODY_SPHERE, (2 * D, 2 * D, 3 * D, D / 2))], tau0,
                       E.BINGHAM if bi > 0 else E.NEWTONIAN)
        st, k, rel = steady_creeping(s, u, p)
        out[f"sphere_box_bi{bi:g}"] = {"C_S": st["drag"] / (6.0 * math.pi * 1.0 * 1.0 * D / 2),
                                      "yield_frac": st["yield_frac"], "steps": k, "last_rel_change": rel,
                                      "cells": n[0] * n[1] * n[2]}
        s.close()
    sph, cube = W.sphere_cube_bodies(D)
    s, u, p = make(n, (W.INFLOW,) * 6, [(E.BODY_SPHERE, sph), (E.BODY_BOX, cube)], W.tau0_for_bingham(10.0, D / 2),
                   E.BINGHAM)
    st, k, rel = steady_creeping(s, u, p)
    lam, dev_ = s.flow_diagnostics(u)
    fluid = s.geometry()["alpha"] > 0
    out["sphere_cube_bi10"] = {"F_D": st["drag"], "yield_frac": st["yield_frac"], "steps": k, "last_rel_change": rel,
                               "lambda_mean": float(lam[fluid].mean()),
                               "unyielded_by_stress_dev": float((dev_[fluid] <= 1e-3).double().mean())}
    s.close()
    out["seconds"] = round(time.perf_counter() - t0, 2)
    return out


def run_adjoint(dev, n=128, steps=40, every=8, advect=0):
    """Drag sensitivities of the step (advect = 0: creeping flow; 1: with the
    convective term): 128^3 sphere channel (r = 0.125, Bi = 5, m = 1e3), a
    seeded Gaussian body force (sigma 0.1), 40 steps at the initial CFL step,
    checkpoints every 8 steps; gradient with respect to tau0, mu and f by the
    adjoint, dJ/dtau0 also by central differences (forward solves to 1e-13)."""
    import torch
    from paper_1905_07392_gb300 import ebvisc
    from paper_1905_07392_gb300 import workloads as W
    w = W.Workload("adjoint_128", n=n, radius=0.125, tau0=W.tau0_for_bingham(5.0, 0.125), m=1e3, seed=3)
    out = {}
    for prec, name in ((ebvisc.FP32_REFINE, "fp32_refine"), (ebvisc.FP64, "fp64")):
        s = ebvisc.Solver.from_workload(w, precision=prec, tol=1e-13, max_iters=20000, advect=advect)
        fluid = (s.geometry()["alpha"] > 0).to(torch.float64)
        u0 = (torch.tensor(W.initial_velocity(w).reshape(3, -1), device=dev) * fluid).reshape(-1).contiguous()
        p0 = torch.zeros(s.nnode, dtype=torch.float64, device=dev)
        f = (torch.tensor(W.body_force(w).reshape(3, -1), device=dev) * fluid).reshape(-1).contiguous()
        dt = s.timestep(u0, f)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, gt, gm, fb = s.drag_gradient(u0, p0, dt, steps, every, f=f)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        entry = {"J": J, "dJ_dtau0": gt, "dJ_dmu": gm, "dJ_df_l2": float(torch.linalg.vector_norm(fb)),
                 "seconds": round(t_adj, 3)}
        if prec == ebvisc.FP32_REFINE:
            def J_of(t):
                s.set_params(tau0=t)
                u, p = u0.clone(), p0.clone()
                acc = 0.0
                for _ in range(steps):
                    acc += s.advance(u, p, dt=dt, f=f, stats=True)["drag"]
                return acc / steps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J0 = J_of(w.tau0)
            t_fwd = time.perf_counter() - t0
            h = 1e-6 * w.tau0
            fd = (J_of(w.tau0 + h) - J_of(w.tau0 - h)) / (2 * h)
            s.set_params(tau0=w.tau0)
            entry.update({"fd_dJ_dtau0": fd, "rel_err_tau0": abs(gt - fd) / abs(fd),
                          "forward_seconds": round(t_fwd, 3),
                          "adjoint_over_forward": round(t_adj / t_fwd, 2), "J_forward": J0})
        out[name] = entry
        s.close()
    form = "full_step" if advect else "creeping"
    out.update({"workload": f"sphere_channel_{n}^3_bi5_m1e3_{form}", "steps": steps, "checkpoint_every": every,
                "dt": dt, "tol": 1e-13})
    return out


def run_batch(dev, world, steps=20, seq_steps=5):
    """The batched sweep: 64 independent instances (N in {48, 64, 96},
    r ~ U[0.08, 0.2], jittered centres, log-uniform Bi in [0.1, 100], m = 1e3),
    FP32 smoother with FP64 refinement to 1e-8, `steps` steps, every step of
    all instances one graph launch.  For comparison the same instances run one
    after another, each from its own captured step graph."""
    import torch
    from paper_1905_07392_gb300 import ebvisc
    from paper_1905_07392_gb300 import workloads as W
    ws = W.batched_sweep()
    t0 = time.perf_counter()
    B = ebvisc.Batch(ws, precision=ebvisc.FP32_REFINE, tol=1e-8, max_iters=2000)
    B.build_spheres()
    setup_s = time.perf_counter() - t0
    us, ps = [], []
    for q, w in enumerate(ws):
        v = B.instance(q)
        alpha = v.geometry()["alpha"]
        u = torch.tensor(W.initial_velocity(w).reshape(3, -1), device=dev)
        us.append((u * (alpha > 0)).reshape(-1).contiguous())
        ps.append(torch.zeros(v.nnode, dtype=torch.float64, device=dev))
    cells = sum(w.n ** 3 for w in ws)
    t0 = time.perf_counter()
    B.advance(us, ps, steps=1, stats=False)          # captures the batch graph
    capture_s = time.perf_counter() - t0
    B.advance(us, ps, steps=2, stats=False)          # warm-up
    torch.cuda.synchronize()
    barrier(world)
    stream = B.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = B.launch_count()
    e0.record(stream)
    B.advance(us, ps, steps=steps, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    sec = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    launches = B.launch_count() - l0
    st = B.advance([u.clone() for u in us], [p.clone() for p in ps], steps=1, stats=True)
    # sequential: each instance's own step graph, one instance after another
    for q in range(len(ws)):
        B.instance(q).advance_graph(us[q], ps[q], steps=1, stats=False)   # capture
    torch.cuda.synchronize()
    e0.record(stream)
    for q in range(len(ws)):
        B.instance(q).advance_graph(us[q], ps[q], steps=seq_steps, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    sec_seq = e0.elapsed_time(e1) / 1e3
    out = {"value": round(cells * steps * world / sec / 1e6, 3), "unit": UNIT,
           "instances": len(ws), "cells_per_step": cells, "steps": steps,
           "sizes": {str(n): sum(1 for w in ws if w.n == n) for n in (48, 64, 96)},
           "ms_per_step": round(1e3 * sec / steps, 3), "graph_launches": steps,
           "gpu_launches": launches, "tol": 1e-8, "precision": "fp32 multigrid, fp64 refinement",
           "max_res_last_step": max(max(x["res"]) for x in st),
           "iters_range_last_step": [min(min(x["iters"]) for x in st), max(max(x["iters"]) for x in st)],
           "sequential_value": round(cells * seq_steps / sec_seq / 1e6, 3),
           "sequential_note": f"{seq_steps} steps per instance, instances one after another",
           "setup_s": round(setup_s, 2), "capture_s": round(capture_s, 2)}
    B.close()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_case(n):
    import numpy as np
    import oracle as O
    from paper_1905_07392_gb300 import workloads as W
    w = workload(256)
    w.n = n
    g = O.Grid(n=(n, n, n), h=1.0 / n)
    geo = O.build_geometry(g, O.Shape(kind=O.SHAPE_SPHERE, p=tuple(w.centre) + (w.radius,)))
    P = O.Params(tau0=w.tau0, m=w.m, bi_cfl=w.bingham, tol=1e-8, model=w.model)
    u = (W.initial_velocity(w).reshape(3, -1) * (geo.alpha > 0)).ravel()
    return O, g, geo, P, u, np.zeros(g.nnode)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def time_oracle(n, steps, warmup):
    """Oracle steps of the benchmark's problem on an n^3 grid: `warmup`
    untimed steps, then `steps` timed; returns (Mcell-steps/s, seconds)."""
    O, g, geo, P, u, p = oracle_case(n)
    for _ in range(warmup):
        u, p, st = O.advance(g, geo, P, u, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        u, p, st = O.advance(g, geo, P, u, p)
    t = time.perf_counter() - t0
    return g.ncell * steps / t / 1e6, t


def cpu_baseline(full=False, n=CPU_SAMPLE_N):
    import oracle as O
    value, t = time_oracle(n, 2, 1)
    out = {"value": round(value, 6), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
           "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
           "sample": f"2 oracle steps (after 1 warm-up) of the same problem (r = 0.1, Bi = 10, m = 1e4, "
                     f"tol 1e-8) on a {n}^3 grid, FP64 C++ with OpenMP on {O.threads()} threads, "
                     f"{t:.1f} s"}
    if full:
        v128, t128 = time_oracle(128, 2, 1)
        out["oracle_128"] = {"value": round(v128, 6), "unit": UNIT, "seconds": round(t128, 1),
                             "sample": "2 oracle steps after 1 warm-up on the 128^3 grid"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle as O
    n = args.cpu_sample_n
    O_, g, geo, P, u, p = oracle_case(n)
    for _ in range(args.warmup):
        u, p, st = O.advance(g, geo, P, u, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, p, st = O.advance(g, geo, P, u, p)
    t = time.perf_counter() - t0
    value = g.ncell * args.steps / t / 1e6
    sample = (f"each step: one oracle step of the same problem on a {n}^3 grid "
              f"(FP64 C++, OpenMP on {O.threads()} threads, tol 1e-8)")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sphere_channel_256^3_bi10_m1e4 (oracle sample {n}^3)"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    rank, world, local = dist_init(args)
    out = run_ours(args, rank, world, local)
    if rank == 0:
        if not args.skip_cpu and world == 1:
            out["cpu_baseline"] = cpu_baseline(full=args.cpu_full, n=args.cpu_sample_n)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

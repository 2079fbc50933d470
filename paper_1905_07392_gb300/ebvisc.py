"""Thin ctypes binding of ``libebvisc.so`` (C-ABI in ``include/ebvisc.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Field arguments are contiguous float64 CUDA tensors (device
pointers are passed through); the library queues its work on the CUDA stream
that was current when the ``Solver`` was created.  There is no CPU fallback:
if the library is missing or fails to load, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libebvisc.so")

INFLOW, OUTFLOW, SLIP, NOSLIP = 0, 1, 2, 3
NEWTONIAN, BINGHAM, HERSCHEL_BULKLEY, POWER_LAW, SOUZA_MENDES_DUTRA = 0, 1, 2, 3, 4
FP64, FP32_REFINE, FP32_MIXED = 0, 1, 2
STATUS = {0: "EBV_OK", -1: "EBV_ERR_INVALID", -2: "EBV_ERR_CUDA", -3: "EBV_ERR_NOT_CONVERGED",
          -4: "EBV_ERR_TIMEOUT", -5: "EBV_ERR_NAN", -6: "EBV_ERR_GEOMETRY", -8: "EBV_ERR_OOM"}


class EbvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("lo", C.c_double * 3), ("h", C.c_double),
                ("bc", C.c_int * 6), ("u_in", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("tau0", C.c_double),
                ("m", C.c_double), ("n_flow", C.c_double), ("eta0", C.c_double),
                ("model", C.c_int), ("cfl", C.c_double), ("bi_cfl", C.c_double),
                ("tol", C.c_double), ("max_iters", C.c_int), ("delta_min", C.c_double),
                ("precision", C.c_int), ("advect", C.c_int)]


class _Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", C.c_double * 6)]


BODY_SPHERE, BODY_BOX, BODY_CYLINDER = 0, 1, 2


class _Stats(C.Structure):
    _fields_ = [("dt", C.c_double), ("drag", C.c_double), ("yield_frac", C.c_double),
                ("iters", C.c_int * 10), ("res", C.c_double * 10), ("div_rel", C.c_double),
                ("ms", C.c_float * 8)]


PHASES = ("timestep", "predictor_derived", "predictor_viscous", "predictor_projection",
          "corrector_derived", "corrector_viscous", "corrector_projection", "drag")


IMPLICIT_FN = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_void_p)

EXPORTS = ["ebv_create", "ebv_set_params", "ebv_build_geometry", "ebv_build_geometry_sphere",
           "ebv_build_geometry_plane", "ebv_get_geometry", "ebv_update_viscosity", "ebv_flow_diagnostics",
           "ebv_derived",
           "ebv_face_states", "ebv_solve_mac", "ebv_solve_viscous", "ebv_solve_projection",
           "ebv_timestep", "ebv_advance", "ebv_advance_graph", "ebv_advance_host", "ebv_drag", "ebv_launch_count",
           "ebv_profile_begin", "ebv_profile_end", "ebv_profile_entry", "ebv_last_error",
           "ebv_destroy", "ebv_drag_noalloc", "ebv_batch_create", "ebv_batch_build_spheres",
           "ebv_batch_instance", "ebv_batch_advance", "ebv_batch_launch_count",
           "ebv_batch_last_error", "ebv_batch_destroy", "ebv_adjoint_step", "ebv_drag_adjoint",
           "ebv_drag_gradient_workspace", "ebv_drag_gradient", "ebv_set_alloc_limit",
           "ebv_set_spin_limit", "ebv_set_fused_sweep", "ebv_set_inner_drop", "ebv_sweep_timing",
           "ebv_save_state", "ebv_load_state", "ebv_build_geometry_spheres",
           "ebv_build_geometry_bodies"]

_lib = None


_variants = {}


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open(path)
    return _lib


def load_variant(path: str):
    """A build variant of the library (same C-ABI, e.g. the FP32-face V-cycle
    of build_lib.VARIANT_LIB) for Solver(..., lib=...); loaded once per path."""
    if path not in _variants:
        _variants[path] = _open(path)
    return _variants[path]


def _open(path):
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "ebv_create": ([C.POINTER(_Grid), C.POINTER(_Params), vp, C.POINTER(vp)], C.c_int),
        "ebv_set_params": ([vp, C.POINTER(_Params)], C.c_int),
        "ebv_build_geometry": ([vp, IMPLICIT_FN, vp], C.c_int),
        "ebv_build_geometry_sphere": ([vp, dp, C.c_double], C.c_int),
        "ebv_build_geometry_plane": ([vp, dp, C.c_double], C.c_int),
        "ebv_get_geometry": ([vp] + [vp] * 8, C.c_int),
        "ebv_update_viscosity": ([vp, vp, vp, vp], C.c_int),
        "ebv_flow_diagnostics": ([vp, vp, vp, vp], C.c_int),
        "ebv_derived": ([vp, vp, vp, vp, vp, ip, dp], C.c_int),
        "ebv_face_states": ([vp, vp, vp], C.c_int),
        "ebv_solve_mac": ([vp, vp, vp, ip, dp], C.c_int),
        "ebv_solve_viscous": ([vp, vp, vp, C.c_double, vp, C.POINTER(_Stats)], C.c_int),
        "ebv_solve_projection": ([vp, vp, vp, C.c_double, C.POINTER(_Stats)], C.c_int),
        "ebv_timestep": ([vp, vp, vp, dp], C.c_int),
        "ebv_advance": ([vp, vp, vp, C.c_double, vp, C.POINTER(_Stats)], C.c_int),
        "ebv_advance_graph": ([vp, vp, vp, C.c_double, vp, C.c_int, C.POINTER(_Stats)], C.c_int),
        "ebv_advance_host": ([vp, vp, vp, C.c_int, C.c_double, C.POINTER(_Stats)], C.c_int),
        "ebv_drag": ([vp, vp, vp, dp, dp], C.c_int),
        "ebv_launch_count": ([vp], C.c_longlong),
        "ebv_profile_begin": ([vp], C.c_int),
        "ebv_profile_end": ([vp, ip], C.c_int),
        "ebv_profile_entry": ([vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong), dp,
                               dp], C.c_int),
        "ebv_last_error": ([vp], C.c_char_p),
        "ebv_destroy": ([vp], None),
        "ebv_drag_noalloc": ([C.POINTER(_Grid), C.POINTER(_Params)] + [vp] * 6 + [C.c_int]
                             + [vp] * 4, C.c_int),
        "ebv_batch_create": ([C.c_int, C.POINTER(_Grid), C.POINTER(_Params), vp, C.POINTER(vp)],
                             C.c_int),
        "ebv_batch_build_spheres": ([vp, dp], C.c_int),
        "ebv_batch_instance": ([vp, C.c_int], vp),
        "ebv_batch_advance": ([vp, C.POINTER(vp), C.POINTER(vp), C.c_int, C.POINTER(_Stats)],
                              C.c_int),
        "ebv_batch_launch_count": ([vp], C.c_longlong),
        "ebv_batch_last_error": ([vp], C.c_char_p),
        "ebv_batch_destroy": ([vp], None),
        "ebv_adjoint_step": ([vp, vp, vp, C.c_double, vp, vp, vp, vp, dp], C.c_int),
        "ebv_drag_adjoint": ([vp, vp, vp, C.c_double, vp, vp, dp], C.c_int),
        "ebv_drag_gradient_workspace": ([vp, C.c_int, C.c_int, C.POINTER(C.c_longlong)], C.c_int),
        "ebv_drag_gradient": ([vp, vp, vp, vp, C.c_double, C.c_int, C.c_int, vp, dp, dp, vp], C.c_int),
        "ebv_set_alloc_limit": ([C.c_longlong], None),
        "ebv_set_spin_limit": ([C.c_longlong], None),
        "ebv_set_fused_sweep": ([C.c_int], None),
        "ebv_set_inner_drop": ([C.c_double], None),
        "ebv_sweep_timing": ([vp, C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
        "ebv_save_state": ([vp, vp, vp, C.c_char_p], C.c_int),
        "ebv_build_geometry_spheres": ([vp, C.c_int, dp], C.c_int),
        "ebv_build_geometry_bodies": ([vp, C.c_int, C.POINTER(_Body)], C.c_int),
        "ebv_load_state": ([vp, vp, vp, C.c_char_p], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("fields must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _check_f64(t, n, name):
    import torch
    if t.dtype != torch.float64 or t.numel() != n:
        raise ValueError(f"{name}: expected {n} float64 values, got {t.numel()} {t.dtype}")


STATUS[-7] = "EBV_ERR_TOO_LARGE"
STATUS[-9] = "EBV_ERR_CUDA_PENDING"


def _check_noalloc_args(grid, geometry, cut, u, p, out):
    """Sizes and types of ebv_drag_noalloc's buffers.  The C entry sees only
    pointers, so this is the one place where a short or mistyped buffer (which
    the kernels would read or write past its end) is refused."""
    import torch
    n = [int(v) for v in grid.n]
    n3 = n[0] * n[1] * n[2]
    nn = (n[0] + 1) * (n[1] + 1) * (n[2] + 1)
    _check_f64(out, 2, "out")
    _check_f64(u, 3 * n3, "u")
    _check_f64(p, nn, "p")
    for name, size in (("alpha", n3), ("area", n3), ("nrm", 3 * n3), ("bcen", 3 * n3)):
        _check_f64(geometry[name], size, name)
    fl = geometry["flag"]
    if fl.dtype != torch.uint8 or fl.numel() != n3:
        raise ValueError(f"flag: expected {n3} uint8 values, got {fl.numel()} {fl.dtype}")
    if cut.dtype != torch.int32:
        raise ValueError("cut must be int32")
    if cut.numel() > n3:
        raise ValueError(f"cut: {cut.numel()} entries for {n3} cells")
    if cut.numel() and (int(cut.min()) < 0 or int(cut.max()) >= n3):
        raise ValueError(f"cut: entries must lie in [0, {n3})")


def drag_noalloc(solver, geometry, cut, u, p, out, stream=None):
    """Drag and unyielded fraction through ebv_drag_noalloc, which allocates
    no GPU memory (for callers that cannot).  `solver` supplies only the grid
    and parameters (its ``_grid`` and ``_params_c()``; no context is used);
    `geometry` is Solver.geometry(); `cut` an int32 CUDA tensor of the cells
    with flag 2 in ascending order; `out` a float64 CUDA tensor of 2 values
    (F_z, unyielded fraction).  Every buffer's size and type is checked here
    before the call."""
    import torch
    _check_noalloc_args(solver._grid, geometry, cut, u, p, out)
    lib = load()
    st = lib.ebv_drag_noalloc(C.byref(solver._grid), C.byref(solver._params_c()),
                              _ptr(geometry["alpha"]), _ptr(geometry["area"]),
                              _ptr(geometry["nrm"]), _ptr(geometry["bcen"]),
                              _ptr(geometry["flag"]), _ptr(cut) if cut.numel() else None,
                              C.c_int(cut.numel()), _ptr(u), _ptr(p), _ptr(out),
                              C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream))
    if st != 0:
        raise EbvError(st, "ebv_drag_noalloc failed")


def _stats_dict(st):
    return {"dt": st.dt, "drag": st.drag, "yield_frac": st.yield_frac,
            "iters": list(st.iters), "res": list(st.res), "div_rel": st.div_rel,
            "ms": dict(zip(PHASES, [float(v) for v in st.ms]))}


class Solver:
    """One grid, one geometry, one CUDA stream."""

    def __init__(self, n, h, lo=(0.0, 0.0, 0.0), bc=W.CHANNEL_BC, u_in=(0.0, 0.0, 1.0), *,
                 rho=1.0, mu=1.0, tau0=0.0, m=1e3, n_flow=1.0, eta0=1e3, model=BINGHAM,
                 cfl=0.5, bi_cfl=0.0, tol=1e-8, max_iters=1000, delta_min=0.01,
                 precision=FP64, advect=1, stream=None, lib=None):
        import torch
        self._lib = lib if lib is not None else load()
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        g = _Grid()
        g.n[:] = list(self.n)
        g.lo[:] = [float(v) for v in lo]
        g.h = self.h
        g.bc[:] = [int(v) for v in bc]
        g.u_in[:] = [float(v) for v in u_in]
        self._grid = g
        self.params = dict(rho=rho, mu=mu, tau0=tau0, m=m, n_flow=n_flow, eta0=eta0, model=model,
                           cfl=cfl, bi_cfl=bi_cfl, tol=tol, max_iters=max_iters,
                           delta_min=delta_min, precision=precision, advect=advect)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = C.c_void_p()
        st = self._lib.ebv_create(C.byref(g), C.byref(self._params_c()),
                                  C.c_void_p(stream.cuda_stream), C.byref(ctx))
        if st != 0:
            raise EbvError(st, "ebv_create failed")
        self._ctx = ctx
        self._fn_keep = None

    @classmethod
    def from_workload(cls, w: W.Workload, **kw):
        args = dict(rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m, n_flow=w.n_flow, model=w.model,
                    cfl=w.cfl, bi_cfl=w.bingham)
        args.update(kw)
        s = cls((w.n, w.n, w.n), w.h, bc=w.bc, u_in=w.u_in, **args)
        s.build_sphere(w.centre, w.radius)
        return s

    def _params_c(self):
        p = _Params()
        for k, v in self.params.items():
            setattr(p, k, int(v) if k in ("model", "max_iters", "precision", "advect") else float(v))
        return p

    def _ok(self, st):
        if st != 0:
            msg = self._lib.ebv_last_error(self._ctx).decode()
            raise EbvError(st, msg)

    def close(self):
        if getattr(self, "_ctx", None):
            if getattr(self, "_owned", True):
                self._lib.ebv_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # sizes
    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def nnode(self):
        return (self.n[0] + 1) * (self.n[1] + 1) * (self.n[2] + 1)

    def nface(self, d):
        m = list(self.n)
        m[d] += 1
        return m[0] * m[1] * m[2]

    def set_params(self, **kw):
        self.params.update(kw)
        self._ok(self._lib.ebv_set_params(self._ctx, C.byref(self._params_c())))

    # geometry
    def build_sphere(self, centre, radius):
        c = (C.c_double * 3)(*centre)
        self._ok(self._lib.ebv_build_geometry_sphere(self._ctx, c, C.c_double(radius)))

    def build_plane(self, normal, d):
        nv = (C.c_double * 3)(*normal)
        self._ok(self._lib.ebv_build_geometry_plane(self._ctx, nv, C.c_double(d)))

    def build_spheres(self, c_r):
        """Union of spheres, rows (cx, cy, cz, r), built on the device."""
        a = np.ascontiguousarray(c_r, dtype=np.float64).reshape(-1, 4)
        self._ok(self._lib.ebv_build_geometry_spheres(self._ctx, a.shape[0],
                                                      a.ctypes.data_as(C.POINTER(C.c_double))))

    def build_bodies(self, bodies):
        """Union of bodies [(kind, (q0, ...)), ...] (BODY_SPHERE / BODY_BOX /
        BODY_CYLINDER, parameters as in ebvisc.h), built on the device."""
        arr = (_Body * len(bodies))()
        for t, (kind, q) in enumerate(bodies):
            arr[t].kind = int(kind)
            vals = [float(v) for v in q] + [0.0] * (6 - len(q))
            arr[t].q[:] = vals
        self._ok(self._lib.ebv_build_geometry_bodies(self._ctx, len(bodies), arr))

    def build_geometry(self, fn):
        """fn(x: tuple of 3 floats) -> float, > 0 in the fluid (called on the host)."""
        cb = IMPLICIT_FN(lambda x, user: float(fn((x[0], x[1], x[2]))))
        self._fn_keep = cb
        self._ok(self._lib.ebv_build_geometry(self._ctx, cb, None))

    def geometry(self):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        N3 = self.ncell
        out = {"alpha": torch.empty(N3, dtype=torch.float64, device=dev),
               "ax": torch.empty(self.nface(0), dtype=torch.float64, device=dev),
               "ay": torch.empty(self.nface(1), dtype=torch.float64, device=dev),
               "az": torch.empty(self.nface(2), dtype=torch.float64, device=dev),
               "area": torch.empty(N3, dtype=torch.float64, device=dev),
               "nrm": torch.empty(3 * N3, dtype=torch.float64, device=dev),
               "bcen": torch.empty(3 * N3, dtype=torch.float64, device=dev),
               "flag": torch.empty(N3, dtype=torch.uint8, device=dev)}
        self._ok(self._lib.ebv_get_geometry(self._ctx, *[_ptr(out[k]) for k in
                                                          ("alpha", "ax", "ay", "az", "area",
                                                           "nrm", "bcen", "flag")]))
        return out

    # stage operations
    def save_state(self, u, p, path):
        """Grid, parameters, geometry, u and p to a file (ebv_save_state)."""
        _check_f64(u, 3 * self.ncell, "u")
        _check_f64(p, self.nnode, "p")
        self._ok(self._lib.ebv_save_state(self._ctx, _ptr(u), _ptr(p), os.fsencode(path)))

    def load_state(self, u, p, path):
        """Parameters and geometry from a file of save_state (same grid); u and
        p receive the saved fields."""
        _check_f64(u, 3 * self.ncell, "u")
        _check_f64(p, self.nnode, "p")
        self._ok(self._lib.ebv_load_state(self._ctx, _ptr(u), _ptr(p), os.fsencode(path)))

    def flow_diagnostics(self, u, lam=None, stress_dev=None):
        """Per cell: Lambda of Eq. ryovar and the yield-stress deviation
        eta ||g|| / tau0 - 1; returns (lam, stress_dev) (allocated if None)."""
        import torch
        _check_f64(u, 3 * self.ncell, "u")
        if lam is None:
            lam = torch.empty(self.ncell, dtype=torch.float64, device=u.device)
        if stress_dev is None:
            stress_dev = torch.empty(self.ncell, dtype=torch.float64, device=u.device)
        _check_f64(lam, self.ncell, "lam")
        _check_f64(stress_dev, self.ncell, "stress_dev")
        self._ok(self._lib.ebv_flow_diagnostics(self._ctx, _ptr(u), _ptr(lam), _ptr(stress_dev)))
        return lam, stress_dev

    def update_viscosity(self, u, eta, srate=None):
        _check_f64(u, 3 * self.ncell, "u")
        _check_f64(eta, self.ncell, "eta")
        if srate is not None:
            _check_f64(srate, self.ncell, "srate")
        self._ok(self._lib.ebv_update_viscosity(self._ctx, _ptr(u), _ptr(eta), _ptr(srate)))

    def derived(self, u, Cv, eta, V):
        it, res = C.c_int(0), C.c_double(0.0)
        self._ok(self._lib.ebv_derived(self._ctx, _ptr(u), _ptr(Cv), _ptr(eta), _ptr(V),
                                       C.byref(it), C.byref(res)))
        return it.value, res.value

    def face_states(self, u, uf):
        self._ok(self._lib.ebv_face_states(self._ctx, _ptr(u), _ptr(uf)))

    def solve_mac(self, uf, phi):
        it, res = C.c_int(0), C.c_double(0.0)
        self._ok(self._lib.ebv_solve_mac(self._ctx, _ptr(uf), _ptr(phi), C.byref(it),
                                         C.byref(res)))
        return it.value, res.value

    def solve_viscous(self, eta, psi, dt, ut):
        st = _Stats()
        self._ok(self._lib.ebv_solve_viscous(self._ctx, _ptr(eta), _ptr(psi), C.c_double(dt),
                                             _ptr(ut), C.byref(st)))
        return _stats_dict(st)

    def solve_projection(self, ut, p, dt):
        st = _Stats()
        self._ok(self._lib.ebv_solve_projection(self._ctx, _ptr(ut), _ptr(p), C.c_double(dt),
                                                C.byref(st)))
        return _stats_dict(st)

    def timestep(self, u, f=None):
        dt = C.c_double(0.0)
        self._ok(self._lib.ebv_timestep(self._ctx, _ptr(u), _ptr(f), C.byref(dt)))
        return dt.value

    def advance(self, u, p, dt=0.0, f=None, stats=True):
        _check_f64(u, 3 * self.ncell, "u")
        _check_f64(p, self.nnode, "p")
        st = _Stats()
        self._ok(self._lib.ebv_advance(self._ctx, _ptr(u), _ptr(p), C.c_double(dt), _ptr(f),
                                       C.byref(st) if stats else None))
        return _stats_dict(st) if stats else None

    def advance_graph(self, u, p, steps=1, dt=0.0, f=None, stats=True):
        """`steps` steps in place, each one launch of the captured step graph."""
        _check_f64(u, 3 * self.ncell, "u")
        _check_f64(p, self.nnode, "p")
        st = _Stats()
        self._ok(self._lib.ebv_advance_graph(self._ctx, _ptr(u), _ptr(p), C.c_double(dt), _ptr(f),
                                             C.c_int(steps), C.byref(st) if stats else None))
        return _stats_dict(st) if stats else None

    def advance_host(self, u: np.ndarray, p: np.ndarray, steps: int, dt=0.0):
        """Steps from host (numpy, float64, contiguous) buffers, updated in place."""
        for a, n in ((u, 3 * self.ncell), (p, self.nnode)):
            if a.dtype != np.float64 or a.size != n or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffers must be contiguous float64 of the right size")
        st = _Stats()
        self._ok(self._lib.ebv_advance_host(self._ctx, C.c_void_p(u.ctypes.data),
                                            C.c_void_p(p.ctypes.data), C.c_int(steps),
                                            C.c_double(dt), C.byref(st)))
        return _stats_dict(st)

    # adjoint of the step (the form the solver's `advect` selects), fixed dt
    def adjoint_step(self, u, p, dt, u_bar, p_bar, f=None, f_bar=None):
        """Reverse of one step from (u, p): u_bar, p_bar (adjoints of the
        outputs) become the adjoints of the inputs; f_bar += adjoint of f.
        Returns (dJ/dtau0, dJ/dmu) of this step."""
        g = (C.c_double * 2)(0.0, 0.0)
        self._ok(self._lib.ebv_adjoint_step(self._ctx, _ptr(u), _ptr(p), C.c_double(dt), _ptr(f), _ptr(u_bar),
                                            _ptr(p_bar), _ptr(f_bar), g))
        return g[0], g[1]

    def drag_adjoint(self, u, p, w, u_bar, p_bar):
        """u_bar, p_bar += w grad F_z(u, p); returns w (dF_z/dtau0, dF_z/dmu)."""
        g = (C.c_double * 2)(0.0, 0.0)
        self._ok(self._lib.ebv_drag_adjoint(self._ctx, _ptr(u), _ptr(p), C.c_double(w), _ptr(u_bar), _ptr(p_bar),
                                            g))
        return g[0], g[1]

    def drag_gradient(self, u0, p0, dt, steps, every=8, f=None, f_grad=True):
        """Time-averaged drag J over `steps` steps (with or without the
        convective term, per `advect`) from (u0, p0) and (dJ/dtau0, dJ/dmu,
        dJ/df or None), checkpointing every `every`."""
        import torch
        n = C.c_longlong(0)
        self._ok(self._lib.ebv_drag_gradient_workspace(self._ctx, steps, every, C.byref(n)))
        work = torch.empty(n.value, dtype=torch.float64, device=u0.device)
        J = C.c_double(0.0)
        g = (C.c_double * 2)(0.0, 0.0)
        fb = torch.empty_like(u0) if f_grad else None
        self._ok(self._lib.ebv_drag_gradient(self._ctx, _ptr(u0), _ptr(p0), _ptr(f), C.c_double(dt), steps, every,
                                             _ptr(work), C.byref(J), g, _ptr(fb)))
        return J.value, g[0], g[1], fb

    def drag(self, u, p):
        fz, yf = C.c_double(0.0), C.c_double(0.0)
        self._ok(self._lib.ebv_drag(self._ctx, _ptr(u), _ptr(p), C.byref(fz), C.byref(yf)))
        return fz.value, yf.value

    def launch_count(self):
        return int(self._lib.ebv_launch_count(self._ctx))

    def sweep_timing(self, level, kind):
        """(fused, passes) ms of one kind of red-black sweep on a MAC level, as
        timed when the solvers were set up (kinds: 0 from zero, 1 plain,
        2 after the coarse correction, 3 with r.z partials)."""
        f, q = C.c_float(0.0), C.c_float(0.0)
        self._ok(self._lib.ebv_sweep_timing(self._ctx, int(level), int(kind), C.byref(f), C.byref(q)))
        return f.value, q.value

    def profile_begin(self):
        """Time every kernel launch of this context with CUDA events."""
        self._ok(self._lib.ebv_profile_begin(self._ctx))

    def profile_end(self):
        """Per kernel name: launches, summed kernel ms, summed algorithmic bytes."""
        n = C.c_int(0)
        self._ok(self._lib.ebv_profile_end(self._ctx, C.byref(n)))
        out = {}
        for i in range(n.value):
            name, L = C.c_char_p(), C.c_longlong(0)
            ms, by = C.c_double(0.0), C.c_double(0.0)
            self._ok(self._lib.ebv_profile_entry(self._ctx, i, C.byref(name), C.byref(L),
                                                 C.byref(ms), C.byref(by)))
            out[name.value.decode()] = {"launches": int(L.value), "ms": float(ms.value),
                                        "bytes": float(by.value)}
        return out


class Batch:
    """Independent sphere-channel instances (each its own grid, rheology and
    sphere) advanced together: every step of all of them is one launch of a
    graph with one branch per instance (ebv_batch_*)."""

    def __init__(self, workloads, precision=FP32_REFINE, tol=1e-8, max_iters=2000, stream=None):
        import torch
        self._lib = load()
        self.workloads = list(workloads)
        n = len(self.workloads)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        # per instance: a Solver-shaped description (no context of its own)
        self._views = []
        grids = (_Grid * n)()
        params = (_Params * n)()
        for q, w in enumerate(self.workloads):
            v = Solver.__new__(Solver)
            v._lib, v.n, v.h, v.stream, v._fn_keep, v._owned = self._lib, (w.n,) * 3, w.h, stream, None, False
            v.params = dict(rho=w.rho, mu=w.mu, tau0=w.tau0, m=w.m, n_flow=w.n_flow, eta0=1e3,
                            model=w.model, cfl=w.cfl, bi_cfl=w.bingham, tol=tol, max_iters=max_iters,
                            delta_min=0.01, precision=precision, advect=1)
            g = _Grid()
            g.n[:] = [w.n] * 3
            g.lo[:] = [0.0, 0.0, 0.0]
            g.h = w.h
            g.bc[:] = [int(b) for b in w.bc]
            g.u_in[:] = [float(x) for x in w.u_in]
            v._grid = g
            grids[q] = g
            params[q] = v._params_c()
            self._views.append(v)
        b = C.c_void_p()
        st = self._lib.ebv_batch_create(n, grids, params, C.c_void_p(stream.cuda_stream), C.byref(b))
        if st != 0:
            raise EbvError(st, "ebv_batch_create failed")
        self._b = b
        for q, v in enumerate(self._views):
            v._ctx = C.c_void_p(self._lib.ebv_batch_instance(b, q))

    def __len__(self):
        return len(self._views)

    def _ok(self, st):
        if st != 0:
            raise EbvError(st, self._lib.ebv_batch_last_error(self._b).decode())

    def build_spheres(self):
        """Each instance's sphere (centre, radius of its workload)."""
        c_r = np.array([list(w.centre) + [w.radius] for w in self.workloads], dtype=np.float64)
        self._ok(self._lib.ebv_batch_build_spheres(self._b, c_r.ctypes.data_as(C.POINTER(C.c_double))))

    def instance(self, q) -> Solver:
        """Instance q as a Solver (the batch owns its context)."""
        return self._views[q]

    def advance(self, us, ps, steps=1, stats=True):
        n = len(self._views)
        for q, v in enumerate(self._views):
            _check_f64(us[q], 3 * v.ncell, f"u[{q}]")
            _check_f64(ps[q], v.nnode, f"p[{q}]")
        U = (C.c_void_p * n)(*[_ptr(t) for t in us])
        P = (C.c_void_p * n)(*[_ptr(t) for t in ps])
        st = (_Stats * n)()
        self._ok(self._lib.ebv_batch_advance(self._b, U, P, C.c_int(steps), st if stats else None))
        return [_stats_dict(x) for x in st] if stats else None

    def launch_count(self):
        return int(self._lib.ebv_batch_launch_count(self._b))

    def close(self):
        if getattr(self, "_b", None):
            for v in self._views:
                v._ctx = None
            self._lib.ebv_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _drag_objective_class():
    import torch

    class DragObjective(torch.autograd.Function):
        """J(tau0, mu, f) = time-averaged drag of `steps` steps of the solver;
        forward runs ebv_drag_gradient (objective and gradient in one pass),
        backward scales the stored gradient.  The solver runs at the given
        tau0 and mu and gets its own parameters back afterwards."""

        @staticmethod
        def forward(ctx, tau0, mu, f, solver, u0, p0, dt, steps, every):
            saved = {"tau0": solver.params["tau0"], "mu": solver.params["mu"]}
            solver.set_params(tau0=float(tau0), mu=float(mu))
            try:
                J, gt, gm, fb = solver.drag_gradient(u0, p0, dt, steps, every, f=f.detach(),
                                                     f_grad=f.requires_grad)
            finally:
                solver.set_params(**saved)
            ctx.grads = (gt, gm, fb)
            ctx.like = (tau0, mu)
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            gt, gm, fb = ctx.grads
            t, m = ctx.like
            dt_ = torch.as_tensor(gt, dtype=t.dtype, device=t.device) * gJ.to(t.device)
            dm_ = torch.as_tensor(gm, dtype=m.dtype, device=m.device) * gJ.to(m.device)
            df_ = fb * gJ.to(fb.device) if fb is not None else None
            return dt_, dm_, df_, None, None, None, None, None, None

    return DragObjective


_DragObjective = None


def drag_objective(solver, tau0, mu, f, u0, p0, dt, steps, every=8):
    """Differentiable time-averaged drag: tau0, mu (0-dim tensors) and f
    (3 x cells CUDA tensor) may require grad."""
    global _DragObjective
    if _DragObjective is None:
        _DragObjective = _drag_objective_class()
    return _DragObjective.apply(tau0, mu, f, solver, u0, p0, dt, steps, every)

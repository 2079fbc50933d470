"""TEST INFRASTRUCTURE ONLY: ctypes wrapper of the plain FP64 C++ oracle.

The oracle restates the embedded-boundary viscoplastic flow step of
arXiv:1905.07392 on the CPU (see ``ebv_oracle.cpp`` for the passages each
function follows).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebv_oracle.cpp")
_HDR = os.path.join(_HERE, "ebv_oracle.h")
_DUAL = os.path.join(_HERE, "og_dual.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

INFLOW, OUTFLOW, SLIP, NOSLIP = 0, 1, 2, 3
NEWTONIAN, BINGHAM, HB, POWERLAW, SMD = 0, 1, 2, 3, 4
SHAPE_NONE, SHAPE_SPHERE, SHAPE_PLANE, SHAPE_UNION = 0, 1, 2, 3
BODY_SPHERE, BODY_BOX, BODY_CYLINDER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (g++ -O2, OpenMP,
    no floating-point contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR, _DUAL))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("lo", C.c_double * 3), ("h", C.c_double),
                ("bc", C.c_int * 6), ("u_in", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("tau0", C.c_double),
                ("m", C.c_double), ("n_flow", C.c_double), ("eta0", C.c_double),
                ("model", C.c_int), ("cfl", C.c_double), ("bi_cfl", C.c_double),
                ("tol", C.c_double), ("max_iters", C.c_int), ("delta_min", C.c_double),
                ("advect", C.c_int)]


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 8), ("nbody", C.c_int), ("bkind", C.c_int * 16),
                ("bq", C.c_double * 96)]


class _Geom(C.Structure):
    _fields_ = [("alpha", C.c_void_p), ("ax", C.c_void_p), ("ay", C.c_void_p),
                ("az", C.c_void_p), ("area", C.c_void_p), ("nrm", C.c_void_p),
                ("bcen", C.c_void_p), ("flag", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("dt", C.c_double), ("drag", C.c_double), ("yield_frac", C.c_double),
                ("iters", C.c_int * 10), ("res", C.c_double * 10)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.og_phi.restype = C.c_double
        _lib.og_eta_of.restype = C.c_double
        _lib.og_timestep.restype = C.c_double
        _lib.og_wall_dudn.restype = C.c_double
        _lib.og_ncell.restype = C.c_size_t
        _lib.og_nnode.restype = C.c_size_t
        _lib.og_drag_tangent.restype = C.c_int
        _lib.og_threads.restype = C.c_int
    return _lib


def threads() -> int:
    """Threads the oracle runs on."""
    return int(lib().og_threads())


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return C.c_void_p(a.ctypes.data)


@dataclass
class Grid:
    n: tuple = (32, 32, 32)
    lo: tuple = (0.0, 0.0, 0.0)
    h: float = 1.0 / 32
    bc: tuple = (SLIP, SLIP, SLIP, SLIP, INFLOW, OUTFLOW)
    u_in: tuple = (0.0, 0.0, 1.0)

    def c(self):
        g = _Grid()
        g.n[:] = list(self.n)
        g.lo[:] = list(self.lo)
        g.h = self.h
        g.bc[:] = list(self.bc)
        g.u_in[:] = list(self.u_in)
        return g

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

    def cshape(self):
        return (self.n[2], self.n[1], self.n[0])

    def fshape(self, d):
        m = [self.n[2], self.n[1], self.n[0]]
        m[2 - d] += 1
        return tuple(m)

    def nshape(self):
        return (self.n[2] + 1, self.n[1] + 1, self.n[0] + 1)


@dataclass
class Params:
    rho: float = 1.0
    mu: float = 1.0
    tau0: float = 0.0
    m: float = 1e3
    n_flow: float = 1.0
    eta0: float = 1e3
    model: int = BINGHAM
    cfl: float = 0.5
    bi_cfl: float = 0.0
    tol: float = 1e-13
    max_iters: int = 200000
    delta_min: float = 0.01
    advect: int = 1

    def c(self):
        p = _Params()
        for k in ("rho", "mu", "tau0", "m", "n_flow", "eta0", "cfl", "bi_cfl", "tol",
                  "delta_min"):
            setattr(p, k, float(getattr(self, k)))
        p.model = int(self.model)
        p.max_iters = int(self.max_iters)
        p.advect = int(self.advect)
        return p


@dataclass
class Shape:
    kind: int = SHAPE_SPHERE
    p: tuple = (0.5, 0.5, 0.5, 0.125)
    bodies: tuple = ()      # SHAPE_UNION: ((BODY_*, (q0, ...)), ...)

    def c(self):
        s = _Shape()
        s.kind = self.kind
        vals = list(self.p) + [0.0] * (8 - len(self.p))
        s.p[:] = vals
        s.nbody = len(self.bodies)
        for b, (kind, q) in enumerate(self.bodies):
            s.bkind[b] = int(kind)
            for e, v in enumerate(q):
                s.bq[6 * b + e] = float(v)
        return s


@dataclass
class Geometry:
    alpha: np.ndarray
    ax: np.ndarray
    ay: np.ndarray
    az: np.ndarray
    area: np.ndarray
    nrm: np.ndarray
    bcen: np.ndarray
    flag: np.ndarray
    _c: object = field(default=None, repr=False)

    def c(self):
        if self._c is None:
            g = _Geom()
            g.alpha, g.ax, g.ay, g.az = (_p(self.alpha), _p(self.ax), _p(self.ay), _p(self.az))
            g.area, g.nrm, g.bcen, g.flag = (_p(self.area), _p(self.nrm), _p(self.bcen),
                                             _p(self.flag))
            self._c = g
        return self._c


def phi(shape: Shape, x):
    return lib().og_phi(C.byref(shape.c()), (C.c_double * 3)(*x))


def build_geometry(grid: Grid, shape: Shape) -> Geometry:
    N3 = grid.ncell
    geo = Geometry(alpha=np.zeros(N3), ax=np.zeros(grid.nface(0)), ay=np.zeros(grid.nface(1)),
                   az=np.zeros(grid.nface(2)), area=np.zeros(N3), nrm=np.zeros(3 * N3),
                   bcen=np.zeros(3 * N3), flag=np.zeros(N3, dtype=np.uint8))
    lib().og_build_geometry(C.byref(grid.c()), C.byref(shape.c()), C.byref(geo.c()))
    return geo


def eta_of(params: Params, sr: float) -> float:
    return lib().og_eta_of(C.byref(params.c()), C.c_double(sr))


def strain_eta(grid, geo, params, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    eta = np.zeros(grid.ncell)
    sr = np.zeros(grid.ncell)
    lib().og_strain_eta(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u),
                        _p(eta), _p(sr))
    return eta, sr


def flow_diagnostics(grid, geo, params, u):
    """Per cell: Lambda of Eq. ryovar and the yield-stress deviation eta ||g|| / tau0 - 1."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    lam = np.zeros(grid.ncell)
    sdev = np.zeros(grid.ncell)
    lib().og_flow_diagnostics(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u), _p(lam),
                              _p(sdev))
    return lam, sdev


def cell_gradient(grid, geo, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    G = np.zeros(9 * grid.ncell)
    lib().og_cell_gradient(C.byref(grid.c()), C.byref(geo.c()), _p(u), _p(G))
    return G


def cc_apply(grid, coeffs, x):
    extra, bx, by, bz = coeffs
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(grid.ncell)
    lib().og_cc_apply(C.byref(grid.c()), _p(extra), _p(bx), _p(by), _p(bz), _p(x), _p(y))
    return y


def cc_solve(grid, coeffs, b, x0=None, tol=1e-13, max_iters=200000):
    extra, bx, by, bz = coeffs
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(grid.ncell) if x0 is None else np.array(x0, dtype=np.float64)
    res = C.c_double(0.0)
    it = lib().og_cc_solve(C.byref(grid.c()), _p(extra), _p(bx), _p(by), _p(bz), _p(b), _p(x),
                           C.c_double(tol), C.c_int(max_iters), C.byref(res))
    return x, it, res.value


def mac_coeffs(grid, geo):
    out = (np.zeros(grid.ncell), np.zeros(grid.nface(0)), np.zeros(grid.nface(1)),
           np.zeros(grid.nface(2)))
    lib().og_mac_coeffs(C.byref(grid.c()), C.byref(geo.c()), *[_p(a) for a in out])
    return out


def visc_coeffs(grid, geo, params, eta, dt, comp):
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    out = (np.zeros(grid.ncell), np.zeros(grid.nface(0)), np.zeros(grid.nface(1)),
           np.zeros(grid.nface(2)))
    rb = np.zeros(grid.ncell)
    lib().og_visc_coeffs(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(eta),
                         C.c_double(dt), C.c_int(comp), *[_p(a) for a in out], _p(rb))
    return out, rb


def nodal_apply(grid, geo, coef, p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    y = np.zeros(grid.nnode)
    lib().og_nodal_apply(C.byref(grid.c()), C.byref(geo.c()), C.c_double(coef), _p(p), _p(y))
    return y


def nodal_rhs(grid, geo, ut):
    ut = np.ascontiguousarray(ut, dtype=np.float64)
    r = np.zeros(grid.nnode)
    lib().og_nodal_rhs(C.byref(grid.c()), C.byref(geo.c()), _p(ut), _p(r))
    return r


def nodal_solve(grid, geo, coef, b, p0=None, tol=1e-13, max_iters=200000):
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = np.zeros(grid.nnode) if p0 is None else np.array(p0, dtype=np.float64)
    res = C.c_double(0.0)
    it = lib().og_nodal_solve(C.byref(grid.c()), C.byref(geo.c()), C.c_double(coef), _p(b),
                              _p(p), C.c_double(tol), C.c_int(max_iters), C.byref(res))
    return p, it, res.value


def cell_grad_p(grid, p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    gp = np.zeros(3 * grid.ncell)
    lib().og_cell_grad_p(C.byref(grid.c()), _p(p), _p(gp))
    return gp


def face_states(grid, geo, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    uf = np.zeros(grid.nface(0) + grid.nface(1) + grid.nface(2))
    lib().og_face_states(C.byref(grid.c()), C.byref(geo.c()), _p(u), _p(uf))
    return uf


def mac_project(grid, geo, uf, tol=1e-13, max_iters=200000):
    uf = np.array(uf, dtype=np.float64)
    phi_ = np.zeros(grid.ncell)
    res = C.c_double(0.0)
    it = lib().og_mac_project(C.byref(grid.c()), C.byref(geo.c()), _p(uf), _p(phi_),
                              C.c_double(tol), C.c_int(max_iters), C.byref(res))
    return uf, phi_, it, res.value


def convective(grid, geo, u, uf):
    u = np.ascontiguousarray(u, dtype=np.float64)
    uf = np.ascontiguousarray(uf, dtype=np.float64)
    Cv = np.zeros(3 * grid.ncell)
    lib().og_convective(C.byref(grid.c()), C.byref(geo.c()), _p(u), _p(uf), _p(Cv))
    return Cv


def redistribute(grid, geo, DC):
    DC = np.ascontiguousarray(DC, dtype=np.float64)
    D = np.zeros(grid.ncell)
    lib().og_redistribute(C.byref(grid.c()), C.byref(geo.c()), _p(DC), _p(D))
    return D


def viscous_explicit(grid, geo, params, u, eta):
    u = np.ascontiguousarray(u, dtype=np.float64)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    V = np.zeros(3 * grid.ncell)
    lib().og_viscous_explicit(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u),
                              _p(eta), _p(V))
    return V


def wall_dudn(grid, geo, u, cell, comp):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().og_wall_dudn(C.byref(grid.c()), C.byref(geo.c()), _p(u), C.c_int(cell),
                              C.c_int(comp))


def derived(grid, geo, params, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    N3 = grid.ncell
    Cv, V = np.zeros(3 * N3), np.zeros(3 * N3)
    eta, sr = np.zeros(N3), np.zeros(N3)
    st = _Stats()
    lib().og_derived(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u), _p(Cv),
                     _p(eta), _p(V), _p(sr), C.byref(st))
    return Cv, eta, V, sr


def timestep(grid, geo, params, u, f=None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().og_timestep(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u),
                             _p(f))


def viscous_solve(grid, geo, params, eta, psi, dt):
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ut = np.zeros(3 * grid.ncell)
    st = _Stats()
    lib().og_viscous_solve(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(eta),
                           _p(psi), C.c_double(dt), _p(ut), C.byref(st), C.c_int(0))
    return ut, list(st.iters[:3]), list(st.res[:3])


def nodal_project(grid, geo, params, dt, ut, p):
    ut = np.array(ut, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    st = _Stats()
    lib().og_nodal_project(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()),
                           C.c_double(dt), _p(ut), _p(p), C.byref(st), C.c_int(0))
    return ut, p, st.iters[0], st.res[0]


def drag(grid, geo, params, u, p):
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    fz, yf = C.c_double(0.0), C.c_double(0.0)
    lib().og_drag(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u), _p(p),
                  C.byref(fz), C.byref(yf))
    return fz.value, yf.value


def advance(grid, geo, params, u, p, dt=0.0, f=None):
    """One step of Algorithm 1; returns (u_new, p_new, stats dict)."""
    u = np.array(u, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    st = _Stats()
    lib().og_advance(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u), _p(p),
                     C.c_double(dt), _p(f), C.byref(st))
    return u, p, {"dt": st.dt, "drag": st.drag, "yield_frac": st.yield_frac,
                  "iters": list(st.iters), "res": list(st.res)}


def drag_tangent(grid, geo, params, u0, p0, dt, steps, f=None, df=None, dtau0=0.0, dmu=0.0):
    """Time-averaged drag J over `steps` steps at fixed dt and its exact
    directional derivative along (dtau0, dmu, df), by forward-mode dual
    numbers through the whole oracle step.  Returns (J, dJ)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    f = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    df = None if df is None else np.ascontiguousarray(df, dtype=np.float64)
    J, dJ = C.c_double(0.0), C.c_double(0.0)
    rc = lib().og_drag_tangent(C.byref(grid.c()), C.byref(geo.c()), C.byref(params.c()), _p(u0), _p(p0),
                               _p(f), _p(df), C.c_double(dtau0), C.c_double(dmu), C.c_double(dt),
                               C.c_int(steps), C.byref(J), C.byref(dJ))
    if rc != 0:
        raise ValueError("og_drag_tangent: dt must be > 0 and steps >= 1")
    return J.value, dJ.value

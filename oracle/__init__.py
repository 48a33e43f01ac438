"""FP64 CPU oracle of the PPML operator-splitting step (arXiv:1607.01105).

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or calls this
package; the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline leg
are its only users.  The scheme itself is plain C in ``ppml_oracle.c`` (compiled with
``-O2 -ffp-contract=off``); this module marshals numpy arrays to it and adds the
time loop.  Exact solutions used as independent pins live in ``oracle.exact``.

State convention: a dict or tuple of six float64 arrays (rho, m_x, m_y, m_z, rho E,
rho eps), each of shape (nz, ny, nx) (x fastest in memory), interior cells only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppml_oracle.c")
_LIB = os.path.join(_HERE, "libppml_oracle.so")

BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, BC_INFLOW = 0, 1, 2, 4
FIRST_ORDER, VHAT_1PT = 1, 2  # scheme variants (Sec. 1.1 first order; 1-point face velocity)
FIELDS = ("rho", "mx", "my", "mz", "en", "ei")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP contraction off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
             "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 6), ("h", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("vacuum_frac", ctypes.c_double),
                ("rho_mean", ctypes.c_double), ("flags", ctypes.c_int),
                ("inflow", (ctypes.c_double * 6) * 6)]


class Diag(ctypes.Structure):
    _fields_ = [("dt_cfl", ctypes.c_double), ("vmax", ctypes.c_double), ("cmax", ctypes.c_double),
                ("sums", ctypes.c_double * 6), ("n_vacuum", ctypes.c_longlong),
                ("n_keep_e", ctypes.c_longlong), ("n_zero_m", ctypes.c_longlong),
                ("n_nonphys", ctypes.c_longlong)]

    def as_dict(self):
        return {"dt_cfl": self.dt_cfl, "vmax": self.vmax, "cmax": self.cmax,
                "sums": list(self.sums), "n_vacuum": self.n_vacuum, "n_keep_e": self.n_keep_e,
                "n_zero_m": self.n_zero_m, "n_nonphys": self.n_nonphys}


_lib = None
_P6 = ctypes.POINTER(ctypes.c_double) * 6
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_step.argtypes = [ctypes.POINTER(_Desc), _P6, _P6, ctypes.c_void_p,
                                     _dp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Diag)]
        _lib.oracle_step.restype = ctypes.c_int
        _lib.oracle_diagnostics.argtypes = [ctypes.POINTER(_Desc), _P6, ctypes.c_double,
                                            ctypes.POINTER(Diag)]
        _lib.oracle_line_parabolas.argtypes = [_dp, ctypes.c_int, _dp, _dp, _dp, _dp]
        for name in ("oracle_avg_right_part", "oracle_avg_left_part"):
            fn = getattr(_lib, name)
            fn.argtypes = [ctypes.c_double] * 4
            fn.restype = ctypes.c_double
        _lib.oracle_face_riemann.argtypes = [ctypes.c_double] * 9 + [_dp, _dp]
        _lib.oracle_face_lambda.argtypes = [ctypes.c_double] * 5
        _lib.oracle_face_lambda.restype = ctypes.c_double
        _lib.oracle_energy_correction.argtypes = [_dp, ctypes.c_double]
        _lib.oracle_energy_correction.restype = ctypes.c_int
        _lib.oracle_lagrangian_step.argtypes = [ctypes.POINTER(_Desc), _P6, _P6, ctypes.c_double,
                                                ctypes.c_double, ctypes.POINTER(Diag)]
        _lib.oracle_lagrangian_step.restype = ctypes.c_int
        _lib.oracle_face_velocities.argtypes = [ctypes.POINTER(_Desc), _P6, ctypes.c_int, _dp]
        _lib.oracle_face_velocities.restype = ctypes.c_int
    return _lib


@dataclass
class Grid:
    """Problem statement: interior cells, spacing, gamma, boundaries (order -x,+x,-y,+y,-z,+z).
    inflow: {face: six conserved values} for the faces whose bc is BC_INFLOW (their ghost
    cells hold that state)."""
    n: tuple  # (nx, ny, nz)
    h: tuple  # (hx, hy, hz)
    gamma: float
    bc: tuple = (BC_OUTFLOW,) * 6
    cfl: float = 0.2
    vacuum_frac: float = 1e-5
    rho_mean: float = 1.0
    flags: int = 0
    inflow: dict = field(default_factory=dict)

    def desc(self) -> _Desc:
        d = _Desc()
        for a in range(3):
            d.n[a] = int(self.n[a])
            d.h[a] = float(self.h[a])
        for q in range(6):
            d.bc[q] = int(self.bc[q])
        d.gamma = float(self.gamma)
        d.vacuum_frac = float(self.vacuum_frac)
        d.rho_mean = float(self.rho_mean)
        d.flags = int(self.flags)
        for q in range(6):
            if self.bc[q] == BC_INFLOW:
                if q not in self.inflow:
                    raise ValueError(f"face {q} is an inflow face without a prescribed state")
                for f in range(6):
                    d.inflow[q][f] = float(self.inflow[q][f])
        return d


def _as_fields(u, shape):
    out = []
    for f in (u[k] for k in FIELDS) if isinstance(u, dict) else u:
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(shape))
        out.append(a)
    if len(out) != 6:
        raise ValueError("state needs six fields")
    return out


def _ptrs(arrs):
    return _P6(*[a.ctypes.data_as(_dp) for a in arrs])


def step(grid: Grid, u, tau: float, phi=None, want_star: bool = False):
    """One step S0-S11.  Returns (u_next, diag_dict[, u_star])."""
    shape = (grid.n[2], grid.n[1], grid.n[0])
    uin = _as_fields(u, shape)
    uout = [np.empty(shape) for _ in range(6)]
    ustar = [np.empty(shape) for _ in range(6)] if want_star else None
    ph = None
    if phi is not None:
        ph = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(shape))
    dg = Diag()
    d = grid.desc()
    rc = lib().oracle_step(ctypes.byref(d), _ptrs(uin), _ptrs(uout),
                           ctypes.cast(_ptrs(ustar), ctypes.c_void_p) if ustar else None,
                           ph.ctypes.data_as(_dp) if ph is not None else None,
                           float(tau), float(grid.cfl), ctypes.byref(dg))
    if rc != 0:
        raise MemoryError("oracle_step failed to allocate")
    if want_star:
        return uout, dg.as_dict(), ustar
    return uout, dg.as_dict()


def lagrangian_step(grid: Grid, u_star, tau: float):
    """The second half of a step (S4-S11) from a given U*: returns (u_next, diag_dict)."""
    shape = (grid.n[2], grid.n[1], grid.n[0])
    us = _as_fields(u_star, shape)
    uout = [np.empty(shape) for _ in range(6)]
    dg = Diag()
    d = grid.desc()
    rc = lib().oracle_lagrangian_step(ctypes.byref(d), _ptrs(us), _ptrs(uout), float(tau),
                                      float(grid.cfl), ctypes.byref(dg))
    if rc != 0:
        raise MemoryError("oracle_lagrangian_step failed to allocate")
    return uout, dg.as_dict()


def diagnostics(grid: Grid, u) -> dict:
    shape = (grid.n[2], grid.n[1], grid.n[0])
    uin = _as_fields(u, shape)
    dg = Diag()
    d = grid.desc()
    lib().oracle_diagnostics(ctypes.byref(d), _ptrs(uin), float(grid.cfl), ctypes.byref(dg))
    return dg.as_dict()


def cfl_dt(grid: Grid, u) -> float:
    return diagnostics(grid, u)["dt_cfl"]


def mean_density(u) -> float:
    rho = u["rho"] if isinstance(u, dict) else u[0]
    return float(np.mean(np.asarray(rho, dtype=np.float64)))


def run(grid: Grid, u, t_end: float, max_steps: int = 10**7, phi=None, callback=None):
    """Advance to t_end with the CFL step, the last step clipped to land on t_end.
    Returns (u, t, steps, diag of the last step)."""
    t = 0.0
    steps = 0
    u = _as_fields(u, (grid.n[2], grid.n[1], grid.n[0]))
    dg = diagnostics(grid, u)
    while t < t_end and steps < max_steps:
        tau = min(dg["dt_cfl"], t_end - t)
        u, dg = step(grid, u, tau, phi=phi)
        t = t + tau if t + tau < t_end else t_end
        steps += 1
        if callback is not None:
            callback(steps, t, u, dg)
    return u, t, steps, dg


def line_parabolas(q):
    """Parabolas (qL, qR, dq, q6) of cells 2..N-3 of a padded line; other entries NaN."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    N = q.size
    outs = [np.full(N, np.nan) for _ in range(4)]
    lib().oracle_line_parabolas(q.ctypes.data_as(_dp), N, *[o.ctypes.data_as(_dp) for o in outs])
    return tuple(outs)


def avg_right_part(qR, dq, q6, y):
    return lib().oracle_avg_right_part(qR, dq, q6, y)


def avg_left_part(qL, dq, q6, y):
    return lib().oracle_avg_left_part(qL, dq, q6, y)


def face_riemann(rl, rr, pl, pr, vls, vrs, pls, prs, gamma):
    V = ctypes.c_double()
    P = ctypes.c_double()
    lib().oracle_face_riemann(rl, rr, pl, pr, vls, vrs, pls, prs, gamma, ctypes.byref(V),
                              ctypes.byref(P))
    return V.value, P.value


def face_lambda(rl, rr, pl, pr, gamma):
    return lib().oracle_face_lambda(rl, rr, pl, pr, gamma)


def energy_correction(u6, rho_vac):
    a = np.ascontiguousarray(u6, dtype=np.float64).copy()
    code = lib().oracle_energy_correction(a.ctypes.data_as(_dp), rho_vac)
    return a, code


def face_velocities(grid: Grid, u_star, axis: int):
    """S5 alone: the face velocities v hat along `axis` of the state u_star (the 9-point
    template of eq. veltemplate and the sqrt(rho) weights of eq.
    modspaceaveragevelocitylagrange), as the Lagrangian stage forms them.  Returns an
    array of shape (nz, ny, nx) with the axis extended by one: entry c along the axis is
    the face between cells c-1 and c."""
    shape = (grid.n[2], grid.n[1], grid.n[0])
    uin = _as_fields(u_star, shape)
    m = [int(grid.n[0]), int(grid.n[1]), int(grid.n[2])]
    m[axis] += 1
    out = np.empty((m[2], m[1], m[0]))
    d = grid.desc()
    rc = lib().oracle_face_velocities(ctypes.byref(d), _ptrs(uin), int(axis), out.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError("face velocities need an active axis")
    return out


def primitives(grid: Grid, u):
    """(rho, vx, vy, vz, p) of a conserved state."""
    rho, mx, my, mz, en, ei = _as_fields(u, (grid.n[2], grid.n[1], grid.n[0]))
    return rho, mx / rho, my / rho, mz / rho, (grid.gamma - 1.0) * ei

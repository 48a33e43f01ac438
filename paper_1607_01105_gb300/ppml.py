"""Thin ctypes binding of libppml.so (C ABI in include/ppml.h).

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
Device memory and streams come from PyTorch.  If the compiled library is missing this
module raises at import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppml.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

PPML_OK, PPML_E_INVAL, PPML_E_CUDA, PPML_E_NONPHYSICAL, PPML_E_TIMEOUT, PPML_E_NOMEM = range(6)
PPML_F32, PPML_F64 = 0, 1
OUTFLOW, PERIODIC, REFLECT, HALO, INFLOW = 0, 1, 2, 3, 4
HALO_PLANES = 3     # planes behind a halo face (z-slab decomposition)
REDUCE_LEN = 10     # max|v|, max c, six sums, vacuum and non-physical counts
FLAG_NONPHYSICAL, FLAG_DT_ZERO = 1, 2
FIRST_ORDER, VHAT_1PT = 1, 2  # scheme variants (ppml_grid_desc.flags)
EXPORTED = ("ppml_init_grid", "ppml_free_grid", "ppml_cfl_dt", "ppml_step", "ppml_eulerian_stage",
            "ppml_conserved_sums", "ppml_read_diag", "ppml_dt_device", "ppml_batch_init",
            "ppml_batch_step", "ppml_batch_status", "ppml_batch_free", "ppml_last_error",
            "ppml_profile", "ppml_kernel_times", "ppml_step_noalloc", "ppml_step_phi",
            "ppml_poisson_periodic", "ppml_poisson_isolated", "ppml_batch_tune",
            "ppml_batch_set_threads", "ppml_fourier_amplitudes", "ppml_fma_peak",
            "ppml_batch_set_split", "ppml_batch_plan", "ppml_grid_tune", "ppml_grid_set_order",
            "ppml_local_reduce", "ppml_lagrangian_stage", "ppml_apply_reduced")
TILE_ORDERS = 4  # launch orders of the stage kernels' tiles (ppml_grid_tune)
NOALLOC_MAX_CELLS = 262144
POISSON_PRINTED_RHS = 1  # isolated solve with the right-hand side exactly as printed


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double * 3), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("bc", ctypes.c_int * 6), ("dtype", ctypes.c_int),
                ("vacuum_frac", ctypes.c_double), ("t_end", ctypes.c_double), ("flags", ctypes.c_int),
                ("rho_ref", ctypes.c_double), ("inflow", (ctypes.c_double * 6) * 6)]


class State(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * 6), ("lo", ctypes.c_void_p * 5)]


class Diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_next", ctypes.c_double), ("vmax", ctypes.c_double),
                ("cmax", ctypes.c_double), ("sums", ctypes.c_double * 6),
                ("steps", ctypes.c_longlong), ("n_vacuum", ctypes.c_longlong),
                ("n_bad", ctypes.c_longlong), ("flags", ctypes.c_uint)]


_vp = ctypes.c_void_p
_lib.ppml_init_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(State), _vp, ctypes.POINTER(_vp)]
_lib.ppml_free_grid.argtypes = [_vp]
_lib.ppml_cfl_dt.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_step.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(State), ctypes.c_double, _vp]
_lib.ppml_eulerian_stage.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(State), ctypes.c_double, _vp]
_lib.ppml_conserved_sums.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_read_diag.argtypes = [_vp, ctypes.POINTER(Diag), _vp]
_lib.ppml_dt_device.argtypes = [_vp]
_lib.ppml_dt_device.restype = _vp
_lib.ppml_batch_init.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp)]
_lib.ppml_batch_step.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), _vp]
_lib.ppml_batch_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_uint), _vp]
_lib.ppml_batch_free.argtypes = [_vp]
_lib.ppml_last_error.restype = ctypes.c_char_p
_lib.ppml_profile.argtypes = [_vp, ctypes.c_int]
_lib.ppml_step_phi.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(State), _vp, ctypes.c_double, _vp]
_lib.ppml_poisson_periodic.argtypes = [_vp, _vp, _vp, ctypes.c_double, _vp]
_lib.ppml_poisson_isolated.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_uint, _vp]
_lib.ppml_batch_tune.argtypes = [_vp, ctypes.c_void_p * 4, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_batch_set_threads.argtypes = [_vp, ctypes.c_int]
_lib.ppml_batch_set_split.argtypes = [_vp, ctypes.c_int]
_lib.ppml_batch_plan.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]
_lib.ppml_fourier_amplitudes.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_step_noalloc.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(State), ctypes.POINTER(State),
                                   ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
_lib.ppml_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]
_lib.ppml_grid_set_order.argtypes = [_vp, ctypes.c_int]
_lib.ppml_local_reduce.argtypes = [_vp, ctypes.POINTER(State), _vp, _vp]
_lib.ppml_lagrangian_stage.argtypes = [_vp, ctypes.POINTER(State), ctypes.POINTER(State), ctypes.c_double,
                                       _vp, _vp]
_lib.ppml_apply_reduced.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_double, _vp]
_lib.ppml_grid_tune.argtypes = [_vp, ctypes.POINTER(State), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double), _vp]


class PPMLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ppml error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != PPML_OK:
        raise PPMLError(rc, _lib.ppml_last_error().decode())


def lib():
    return _lib


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def torch_dtype(dtype: int):
    return torch.float64 if dtype == PPML_F64 else torch.float32


def _state(fields, dtype=None, shape=None) -> State:
    """Six fields, or eleven: the six and the low parts of rho, m_x, m_y, m_z, rho E of a
    double-float FP32 state."""
    if len(fields) not in (6, 11):
        raise ValueError("a state has six fields (or six and five low parts)")
    s = State()
    for i, t in enumerate(fields):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("state fields must be contiguous CUDA tensors")
        if dtype is not None and t.dtype != dtype:
            raise ValueError(f"field {i} has dtype {t.dtype}, expected {dtype}")
        if shape is not None and t.numel() != shape:
            raise ValueError(f"field {i} has {t.numel()} elements, expected {shape}")
        if i < 6:
            s.f[i] = t.data_ptr()
        else:
            s.lo[i - 6] = t.data_ptr()
    return s


class Grid:
    """Handle over ppml_init_grid / ppml_step / ppml_cfl_dt / ppml_read_diag.
    inflow: {face: six conserved values} for the faces whose bc is INFLOW."""

    def __init__(self, n, h, gamma, cfl, bc=(OUTFLOW,) * 6, dtype=PPML_F32, u0=None,
                 vacuum_frac=1e-5, t_end=0.0, stream=None, flags=0, rho_ref=0.0, inflow=None):
        d = GridDesc()
        d.nx, d.ny, d.nz = (int(x) for x in n)
        for a in range(3):
            d.h[a] = float(h[a])
        d.gamma, d.cfl = float(gamma), float(cfl)
        for q in range(6):
            d.bc[q] = int(bc[q])
        d.dtype = int(dtype)
        d.vacuum_frac = float(vacuum_frac)
        d.t_end = float(t_end)
        d.flags = int(flags)
        d.rho_ref = float(rho_ref)
        inflow = inflow or {}
        for q in range(6):
            if int(bc[q]) == INFLOW:
                if q not in inflow:
                    raise ValueError(f"face {q} is an inflow face without a prescribed state")
                for f in range(6):
                    d.inflow[q][f] = float(inflow[q][f])
        self.desc = d
        self.n = tuple(int(x) for x in n)
        self.cells = self.n[0] * self.n[1] * self.n[2]
        self.dtype = int(dtype)
        self.tdtype = torch_dtype(dtype)
        self._h = ctypes.c_void_p()
        st = u0 if isinstance(u0, State) else _state(u0, self.tdtype, self.cells)
        _check(_lib.ppml_init_grid(ctypes.byref(d), ctypes.byref(st), _stream(stream),
                                   ctypes.byref(self._h)))

    def close(self):
        if self._h:
            _lib.ppml_free_grid(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cfl_dt(self, u, sync=True, stream=None):
        st = _state(u, self.tdtype, self.cells)
        out = ctypes.c_double()
        _check(_lib.ppml_cfl_dt(self._h, ctypes.byref(st), ctypes.byref(out) if sync else None,
                                _stream(stream)))
        return out.value if sync else None

    def step(self, u_in, u_out, dt=0.0, stream=None):
        a = _state(u_in, self.tdtype, self.cells)
        b = _state(u_out, self.tdtype, self.cells)
        _check(_lib.ppml_step(self._h, ctypes.byref(a), ctypes.byref(b), float(dt), _stream(stream)))

    def step_phi(self, u_in, u_out, phi, dt=0.0, stream=None):
        """Step with the gravitational potential phi (device tensor of the grid's dtype)."""
        a = _state(u_in, self.tdtype, self.cells)
        b = _state(u_out, self.tdtype, self.cells)
        if phi is not None and (not phi.is_cuda or phi.dtype != self.tdtype or phi.numel() != self.cells):
            raise ValueError("phi must be a CUDA tensor of the grid's dtype and size")
        _check(_lib.ppml_step_phi(self._h, ctypes.byref(a), ctypes.byref(b),
                                  phi.data_ptr() if phi is not None else None, float(dt), _stream(stream)))

    def poisson_periodic(self, rho, phi, G=1.0, stream=None):
        """Periodic 27-point Poisson solve of rho into phi (device tensors, grid dtype)."""
        for t in (rho, phi):
            if not t.is_cuda or t.dtype != self.tdtype or t.numel() != self.cells or not t.is_contiguous():
                raise ValueError("rho and phi must be contiguous CUDA tensors of the grid's dtype and size")
        _check(_lib.ppml_poisson_periodic(self._h, rho.data_ptr(), phi.data_ptr(), float(G), _stream(stream)))

    def poisson_isolated(self, rho, phi, G=1.0, printed_rhs=False, stream=None):
        """Isolated-boundary 27-point Poisson solve of rho into phi (multipole shell, sine
        transforms); the grid is centred on the origin of the expansion."""
        for t in (rho, phi):
            if not t.is_cuda or t.dtype != self.tdtype or t.numel() != self.cells or not t.is_contiguous():
                raise ValueError("rho and phi must be contiguous CUDA tensors of the grid's dtype and size")
        _check(_lib.ppml_poisson_isolated(self._h, rho.data_ptr(), phi.data_ptr(), float(G),
                                          POISSON_PRINTED_RHS if printed_rhs else 0, _stream(stream)))

    def fourier_amplitudes(self, rho, r_f, m_max=8, stream=None):
        """Global Fourier amplitudes A_1..A_m_max of the column density within r_f of the
        z axis (the grid is centred on the axis).  Synchronizes."""
        if not rho.is_cuda or rho.dtype != self.tdtype or rho.numel() != self.cells or not rho.is_contiguous():
            raise ValueError("rho must be a contiguous CUDA tensor of the grid's dtype and size")
        out = (ctypes.c_double * int(m_max))()
        _check(_lib.ppml_fourier_amplitudes(self._h, rho.data_ptr(), float(r_f), int(m_max), out,
                                            _stream(stream)))
        return list(out)

    def eulerian_stage(self, u_in, u_star, dt, stream=None):
        a = _state(u_in, self.tdtype, self.cells)
        b = _state(u_star, self.tdtype, self.cells)
        _check(_lib.ppml_eulerian_stage(self._h, ctypes.byref(a), ctypes.byref(b), float(dt),
                                        _stream(stream)))

    # z-slab decomposition: the state arguments are State structures (their pointers lead
    # the interior planes of halo-padded arrays); red is a CUDA float64 tensor of REDUCE_LEN
    def local_reduce(self, st, red, stream=None):
        _check(_lib.ppml_local_reduce(self._h, ctypes.byref(st), red.data_ptr(), _stream(stream)))

    def lagrangian_stage(self, st_star, st_out, dt, red, stream=None):
        _check(_lib.ppml_lagrangian_stage(self._h, ctypes.byref(st_star), ctypes.byref(st_out),
                                          float(dt), red.data_ptr(), _stream(stream)))

    def eulerian_stage_ptrs(self, st_in, st_star, dt, stream=None):
        _check(_lib.ppml_eulerian_stage(self._h, ctypes.byref(st_in), ctypes.byref(st_star),
                                        float(dt), _stream(stream)))

    def apply_reduced(self, red, advance, dt=0.0, stream=None):
        _check(_lib.ppml_apply_reduced(self._h, red.data_ptr(), 1 if advance else 0, float(dt),
                                       _stream(stream)))

    def conserved_sums(self, u, stream=None):
        st = _state(u, self.tdtype, self.cells)
        out = (ctypes.c_double * 6)()
        _check(_lib.ppml_conserved_sums(self._h, ctypes.byref(st), out, _stream(stream)))
        return list(out)

    def diag(self, stream=None, raise_nonphysical=True) -> dict:
        d = Diag()
        rc = _lib.ppml_read_diag(self._h, ctypes.byref(d), _stream(stream))
        if rc != PPML_OK and (rc != PPML_E_NONPHYSICAL or raise_nonphysical):
            _check(rc)
        return {"t": d.t, "dt_next": d.dt_next, "vmax": d.vmax, "cmax": d.cmax,
                "sums": list(d.sums), "steps": d.steps, "n_vacuum": d.n_vacuum,
                "n_bad": d.n_bad, "flags": d.flags}

    def set_order(self, order):
        """Launch order of the stage kernels' tiles (0 x-major, 1 z-major, 2 and 3 blocked)."""
        _check(_lib.ppml_grid_set_order(self._h, int(order)))

    def tune(self, u, trial_steps=5, stream=None):
        """Time each tile order on scratch copies of u's fields; keep the fastest.
        Returns (order, {order: ms})."""
        st = _state(u, self.tdtype, self.cells)
        chosen = ctypes.c_int(-1)
        ms = (ctypes.c_double * TILE_ORDERS)()
        _check(_lib.ppml_grid_tune(self._h, ctypes.byref(st), int(trial_steps), ctypes.byref(chosen),
                                   ms, _stream(stream)))
        return chosen.value, dict(enumerate(list(ms)))

    def dt_device_ptr(self) -> int:
        return _lib.ppml_dt_device(self._h)

    def profile(self, enable: bool):
        _check(_lib.ppml_profile(self._h, 1 if enable else 0))

    def kernel_times(self):
        """(ms_eulerian, ms_lagrangian, ms_finalize) accumulated, and the step count."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_longlong()
        _check(_lib.ppml_kernel_times(self._h, ms, ctypes.byref(n)))
        return list(ms), n.value


def make_desc(n, h, gamma, cfl, bc=(OUTFLOW,) * 6, dtype=PPML_F32, vacuum_frac=1e-5, t_end=0.0,
              flags=0, rho_ref=0.0):
    d = GridDesc()
    d.nx, d.ny, d.nz = (int(x) for x in n)
    for a in range(3):
        d.h[a] = float(h[a])
    d.gamma, d.cfl = float(gamma), float(cfl)
    for q in range(6):
        d.bc[q] = int(bc[q])
    d.dtype = int(dtype)
    d.vacuum_frac = float(vacuum_frac)
    d.t_end = float(t_end)
    d.flags = int(flags)
    d.rho_ref = float(rho_ref)
    return d


def step_noalloc(desc, u_in, u_out, dt, rho_mean, stream=None, want_diag=True):
    """ppml_step_noalloc: one step without a handle and without device allocation (for
    callers that cannot allocate).  Returns (dt_next, vmax, cmax, sums[6]) when want_diag."""
    cells = desc.nx * desc.ny * desc.nz
    tdt = torch_dtype(desc.dtype)
    a = _state(u_in, tdt, cells)
    b = _state(u_out, tdt, cells)
    out = (ctypes.c_double * 9)()
    _check(_lib.ppml_step_noalloc(ctypes.byref(desc), ctypes.byref(a), ctypes.byref(b), float(dt),
                                  float(rho_mean), out if want_diag else None, _stream(stream)))
    if not want_diag:
        return None
    return out[0], out[1], out[2], list(out[3:9])


class Batch:
    """Handle over ppml_batch_init / ppml_batch_step / ppml_batch_status."""

    def __init__(self, ncells, h, t_end, gamma, cfl, dtype=PPML_F32, vacuum_frac=1e-5):
        n = len(ncells)
        self.n_inst = n
        self.dtype = int(dtype)
        self.tdtype = torch_dtype(dtype)
        self.total = int(sum(int(x) for x in ncells))
        nc = (ctypes.c_int * n)(*[int(x) for x in ncells])
        hh = (ctypes.c_double * n)(*[float(x) for x in h])
        te = (ctypes.c_double * n)(*[float(x) for x in t_end])
        self._h = ctypes.c_void_p()
        _check(_lib.ppml_batch_init(n, nc, hh, te, float(gamma), float(cfl), float(vacuum_frac),
                                    self.dtype, ctypes.byref(self._h)))

    def _ptrs(self, fields):
        if len(fields) != 4:
            raise ValueError("a batch state has four fields")
        ptrs = (ctypes.c_void_p * 4)()
        for i, t in enumerate(fields):
            if not t.is_cuda or not t.is_contiguous() or t.dtype != self.tdtype or t.numel() != self.total:
                raise ValueError(f"batch field {i} has the wrong device, layout, dtype or size")
            ptrs[i] = t.data_ptr()
        return ptrs

    def tune(self, fields, trial_steps=20, stream=None):
        """Time the CTA sizes 256/512/1024 on scratch copies of `fields`; keep the fastest.
        Returns (threads, {threads: ms})."""
        ptrs = self._ptrs(fields)
        chosen = ctypes.c_int(0)
        ms = (ctypes.c_double * 3)()
        _check(_lib.ppml_batch_tune(self._h, ptrs, int(trial_steps), ctypes.byref(chosen), ms,
                                    _stream(stream)))
        return chosen.value, dict(zip((256, 512, 1024), list(ms)))

    def set_split(self, min_cells):
        """Instances of at least min_cells cells take a CTA pair (0: none)."""
        _check(_lib.ppml_batch_set_split(self._h, int(min_cells)))

    def set_threads(self, threads):
        _check(_lib.ppml_batch_set_threads(self._h, int(threads)))

    def step(self, fields, max_steps, sync=False, stream=None, lo=None):
        """Advance the batch; `lo`: None or three tensors with the low parts of rho, m,
        rho E (FP32).  With sync, returns the number of instances at their end time."""
        ptrs = self._ptrs(fields)
        lptr = None
        if lo is not None:
            if len(lo) != 3:
                raise ValueError("three low-part arrays")
            lptr = (ctypes.c_void_p * 3)()
            for i, t in enumerate(lo):
                if not t.is_cuda or not t.is_contiguous() or t.dtype != self.tdtype or t.numel() != self.total:
                    raise ValueError(f"low part {i} has the wrong device, layout, dtype or size")
                lptr[i] = t.data_ptr()
        done = ctypes.c_int(-1)
        _check(_lib.ppml_batch_step(self._h, ptrs, lptr, int(max_steps),
                                    ctypes.byref(done) if sync else None, _stream(stream)))
        return done.value if sync else None

    def status(self, stream=None, with_flags=False):
        """(t, steps) per instance, and with_flags also the flags (PPML_FLAG_NONPHYSICAL);
        a flagged instance does not raise here."""
        t = (ctypes.c_double * self.n_inst)()
        s = (ctypes.c_int * self.n_inst)()
        fl = (ctypes.c_uint * self.n_inst)()
        rc = _lib.ppml_batch_status(self._h, t, s, fl, _stream(stream))
        if rc != PPML_OK and rc != PPML_E_NONPHYSICAL:
            _check(rc)
        if with_flags:
            return list(t), list(s), list(fl)
        return list(t), list(s)

    def close(self):
        if self._h:
            _lib.ppml_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_plan(ncells, split_min):
    """Work plan of ppml_batch_plan: (items as a list of (a, b), order or None)."""
    n = len(ncells)
    cells = (ctypes.c_int * n)(*[int(x) for x in ncells])
    items = (ctypes.c_int * (2 * n))()
    order = (ctypes.c_int * n)()
    k = ctypes.c_int()
    _check(_lib.ppml_batch_plan(n, cells, int(split_min), items, ctypes.byref(k), order))
    if k.value == 0:
        return [], list(order)
    return [(items[2 * i], items[2 * i + 1]) for i in range(k.value)], None


def fma_peak(dtype: int, iters: int, stream=None) -> float:
    """Measured FMAs per second of the device for PPML_F32 or PPML_F64 (ppml_fma_peak)."""
    out = ctypes.c_double()
    _check(_lib.ppml_fma_peak(int(dtype), int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


def to_device(u, dtype: int, device="cuda", lo=False):
    """Six (or four) float64 numpy arrays -> contiguous CUDA tensors of the path's dtype.
    lo (FP32): append the low parts of the first n - 1 fields (rho, m..., rho E), so that
    hi + lo holds the FP64 input to about 48 bits: a double-float state."""
    t = [torch.as_tensor(a).to(device=device, dtype=torch.float64).contiguous().reshape(-1) for a in u]
    hi = [x.to(torch_dtype(dtype)) for x in t]
    if not lo:
        return hi
    if dtype != PPML_F32:
        raise ValueError("low parts are for FP32 states")
    return hi + [(x - h.double()).float() for x, h in zip(t[:-1], hi[:-1])]


def value_of(state, f):
    """Field f of a state as float64 (hi + lo for a double-float state)."""
    x = state[f].double()
    if len(state) == 11 and f < 5:
        x = x + state[6 + f].double()
    elif len(state) == 7 and f < 3:  # batch: rho, m, rho E, rho eps + 3 low parts
        x = x + state[4 + f].double()
    return x

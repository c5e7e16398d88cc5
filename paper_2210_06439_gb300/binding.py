"""Thin ctypes binding of the C ABI in include/oct_hydro.h.

Argument marshalling only: every step of the hydro path runs in the CUDA
library.  Functions keep the C names; ``Hydro`` wraps a handle for callers
holding torch CUDA tensors.  Importing this module loads liboct_hydro.so and
raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OCT_OK, OCT_E_ARG, OCT_E_CUDA, OCT_E_NONPHYS, OCT_E_TIMEOUT, OCT_E_NOMEM, OCT_E_STATE = 0, -1, -2, -3, -4, -5, -6
OCT_FP64, OCT_MIXED = 0, 1
OCT_BC_GIVEN, OCT_BC_PERIODIC, OCT_BC_OUTFLOW, OCT_BC_AMR = 0, 1, 2, 3
OCT_RECON_CONSERVED, OCT_RECON_PRIMITIVE = 0, 1
OCT_FLAG_NONPHYS, OCT_FLAG_FLOOR, OCT_FLAG_NO_SOURCE = 0x1, 0x2, 0x4

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64

# name -> (restype, argtypes); the declarations of include/oct_hydro.h
SIGNATURES = {
    "oct_hydro_create": (_I, [_I, _I, _I, _I, _D, ctypes.POINTER(_P)]),
    "oct_hydro_set_layout": (_I, [_P, _P, _P, _P, _P, _P, _I]),
    "oct_hydro_set_amr": (_I, [_P, _P, _P, _I, _I]),
    "oct_hydro_set_reconstruction": (_I, [_P, _I]),
    "oct_hydro_set_prolongation": (_I, [_P, _I]),
    "oct_hydro_set_params": (_I, [_P, _I, _D, _D, _D, _D]),
    "oct_hydro_set_dt_cap": (_I, [_P, _D]),
    "oct_hydro_state_len": (_I64, [_P]),
    "oct_hydro_rhs_len": (_I64, [_P]),
    "oct_hydro_rhs": (_I, [_P, _P, _P, _P, _P]),
    "oct_hydro_max_dt": (_I, [_P, _P, _P, _P]),
    "oct_hydro_fill_ghosts": (_I, [_P, _P, _P]),
    "oct_hydro_rk_step": (_I, [_P, _P, _P, _P]),
    "oct_hydro_rk_steps_host": (_I, [_P, _P, _I, _P, _P]),
    "oct_hydro_rhs_host": (_I, [_P, _P, _P, _P]),
    "oct_hydro_autotune": (_I, [_P, _P, _P]),
    "oct_hydro_rhs_dt_noalloc": (_I, [_I, _I, _I, _D, _I, _D, _D, _P, _P, _P, _P, _P]),
    "oct_hydro_launch_info": (_I, [_P, _P, _P, _P]),
    "oct_hydro_step_launches": (_I, [_P]),
    "oct_hydro_host_copy_bytes": (_I, [_P, _P, _P]),
    "oct_hydro_gravity_monopole": (_I, [_P, _P, _D, _D, _P, _P, _P]),
    "oct_hydro_pipe_peaks": (_I, [_D, _P, _P, _P]),
    "oct_hydro_eval_math": (_I, [_I, _P, _P, _I64, _D, _P]),
    "oct_hydro_get_error_flags": (_I, [_P, _P]),
    "oct_hydro_last_error": (ctypes.c_char_p, []),
    "oct_hydro_destroy": (None, [_P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads liboct_hydro.so (building it first when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class OctError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"oct_hydro status {status}: {msg}")
        self.status = status


def check(status):
    if status != OCT_OK:
        raise OctError(status, load().oct_hydro_last_error().decode())
    return status


def _ptr(x):
    """Device or host address of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def pipe_peaks(target_ms=200.0, stream=None):
    """(FP64, FP32) FMA throughput of the current GPU in TFLOP/s (an FMA
    counts as two flops), each from one launch of at least target_ms."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    check(load().oct_hydro_pipe_peaks(float(target_ms), ctypes.addressof(f64), ctypes.addressof(f32),
                                      _stream_ptr(stream)))
    return f64.value, f32.value


def eval_math(which, x, y, gamma=5.0 / 3.0, stream=None):
    """y = fn(x) elementwise on device float64 tensors (oct_hydro_eval_math)."""
    check(load().oct_hydro_eval_math(int(which), _ptr(x), _ptr(y), int(x.numel()), float(gamma),
                                     _stream_ptr(stream)))


class Hydro:
    """Owns one oct_hydro handle.  Tensors are torch CUDA float64 tensors
    (state in the library's ghosted layout, dUdt in the RHS layout)."""

    def __init__(self, n_subgrids, edge, n_species, gamma=5.0 / 3.0, ghost=3):
        L = load()
        h = _P()
        check(L.oct_hydro_create(int(n_subgrids), int(edge), int(ghost), int(n_species), float(gamma),
                                 ctypes.byref(h)))
        self.h = h
        self.L = L
        self.n_subgrids = int(n_subgrids)

    @classmethod
    def from_problem(cls, prob, precision=OCT_FP64, cfl=0.4, rho_floor=1e-12, eps1=1e-3, eps2=0.1,
                     recon=OCT_RECON_CONSERVED):
        """Handle for an ``inputs.Problem`` (layout copied from it)."""
        edges = np.ascontiguousarray(prob.edge, np.int32)
        uniform = bool(np.all(edges == edges[0]))
        self = cls(prob.n_sub, int(edges[0]) if uniform else 0, prob.n_species, prob.gamma)
        self.set_layout(edges, prob.off, prob.dx, prob.level, prob.nbr, prob.bc if prob.bc != OCT_BC_AMR else 0)
        if prob.bc == OCT_BC_AMR:
            m = prob.meta
            self.set_amr(m["level"], m["origin"], m["n0"], m["periodic"])
        self.set_params(precision, cfl, rho_floor, eps1, eps2)
        if recon != OCT_RECON_CONSERVED:
            self.set_reconstruction(recon)
        return self

    def close(self):
        if getattr(self, "h", None):
            self.L.oct_hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layout(self, edges, offsets, dx, level=None, neighbours=None, bc=OCT_BC_GIVEN):
        self._keep = [np.ascontiguousarray(edges, np.int32), np.ascontiguousarray(offsets, np.int64),
                      np.ascontiguousarray(dx, np.float64),
                      None if level is None else np.ascontiguousarray(level, np.int32),
                      None if neighbours is None else np.ascontiguousarray(neighbours, np.int32)]
        e, o, d, l, n = self._keep
        check(self.L.oct_hydro_set_layout(self.h, e.ctypes.data, o.ctypes.data, d.ctypes.data,
                                          None if l is None else l.ctypes.data,
                                          None if n is None else n.ctypes.data, int(bc)))

    def set_amr(self, level, origin, root_cells, periodic=True):
        self._amr = [np.ascontiguousarray(level, np.int32), np.ascontiguousarray(origin, np.int32).reshape(-1)]
        check(self.L.oct_hydro_set_amr(self.h, self._amr[0].ctypes.data, self._amr[1].ctypes.data, int(root_cells),
                                       int(bool(periodic))))

    def set_prolongation(self, order):
        check(self.L.oct_hydro_set_prolongation(self.h, int(order)))

    def set_reconstruction(self, variables):
        check(self.L.oct_hydro_set_reconstruction(self.h, int(variables)))

    def set_params(self, precision=OCT_FP64, cfl=0.4, rho_floor=1e-12, eps1=1e-3, eps2=0.1):
        check(self.L.oct_hydro_set_params(self.h, int(precision), float(cfl), float(rho_floor), float(eps1),
                                          float(eps2)))

    def set_dt_cap(self, dt_cap):
        check(self.L.oct_hydro_set_dt_cap(self.h, float(dt_cap)))

    @property
    def state_len(self):
        return int(self.L.oct_hydro_state_len(self.h))

    @property
    def rhs_len(self):
        return int(self.L.oct_hydro_rhs_len(self.h))

    def rhs(self, U, dUdt, amax=None, stream=None):
        check(self.L.oct_hydro_rhs(self.h, _ptr(U), _ptr(dUdt), _ptr(amax), _stream_ptr(stream)))

    def max_dt(self, U, stream=None):
        out = ctypes.c_double()
        check(self.L.oct_hydro_max_dt(self.h, _ptr(U), ctypes.addressof(out), _stream_ptr(stream)))
        return out.value

    def fill_ghosts(self, U, stream=None):
        check(self.L.oct_hydro_fill_ghosts(self.h, _ptr(U), _stream_ptr(stream)))

    def rk_step(self, U, want_dt=True, stream=None):
        out = ctypes.c_double()
        check(self.L.oct_hydro_rk_step(self.h, _ptr(U), ctypes.addressof(out) if want_dt else None,
                                       _stream_ptr(stream)))
        return out.value if want_dt else None

    def rk_steps_host(self, U_host, n_steps=1, stream=None):
        out = ctypes.c_double()
        check(self.L.oct_hydro_rk_steps_host(self.h, _ptr(U_host), int(n_steps), ctypes.addressof(out),
                                             _stream_ptr(stream)))
        return out.value

    def rhs_host(self, U_host, dUdt_host, stream=None):
        check(self.L.oct_hydro_rhs_host(self.h, _ptr(U_host), _ptr(dUdt_host), _stream_ptr(stream)))

    def gravity_monopole(self, U, phi, g, G=1.0, r_s=2.0 / 0.34, stream=None):
        """Same-level monopole gravity of the state U into phi [n * E^3] and
        g [n * 3 * E^3] (device float64 tensors)."""
        check(self.L.oct_hydro_gravity_monopole(self.h, _ptr(U), float(G), float(r_s), _ptr(phi), _ptr(g),
                                                _stream_ptr(stream)))

    def autotune(self, U, stream=None):
        check(self.L.oct_hydro_autotune(self.h, _ptr(U), _stream_ptr(stream)))

    def launch_info(self):
        """(tile mode, CTAs per SM, work items) of the RHS launch."""
        t, c, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self.L.oct_hydro_launch_info(self.h, ctypes.addressof(t), ctypes.addressof(c), ctypes.addressof(n)))
        return t.value, c.value, n.value

    def host_copy_bytes(self):
        """(host-to-device, device-to-host) bytes of one rk_steps_host call."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        check(self.L.oct_hydro_host_copy_bytes(self.h, ctypes.addressof(a), ctypes.addressof(b)))
        return a.value, b.value

    def step_launches(self):
        """Kernel launches of one rk_step for the current layout."""
        n = self.L.oct_hydro_step_launches(self.h)
        if n < 0:
            raise OctError(OCT_E_STATE, "no layout")
        return n

    def tile_mode(self):
        return self.launch_info()[0]

    def error_flags(self):
        v = ctypes.c_uint32()
        check(self.L.oct_hydro_get_error_flags(self.h, ctypes.addressof(v)))
        return int(v.value)

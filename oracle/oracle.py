"""ctypes binding of the C oracle in ``oct_oracle.c`` (test infrastructure only).

The C file is compiled with ``gcc -O2 -ffp-contract=off`` so that each
floating-point operation is a single IEEE round-to-nearest FP64 operation
(no FMA contraction).  OpenMP parallelises over independent subgrids only,
which leaves every result bit-identical to the single-threaded build.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oct_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboct_oracle.so")

__all__ = [
    "build_oracle", "lib", "ppm", "prim", "kt_point", "simpson", "rhs", "rhs_cells",
    "dt_from_amax", "ghost_fill", "floors", "rk_combine", "rk3_step", "max_threads", "amr_ghost_fill",
    "rk3_step_amr", "rhs_faces", "amr_reflux", "gravity_monopole",
]

_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared",
            "-Wall", "-Wno-unknown-pragmas"]
    tmp = _OUT + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True, text=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        _declare(_lib)
    return _lib


_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def _declare(L):
    L.oco_gravity_monopole.argtypes = [_I, _I, _P, _I, _P, _D, _D, _D, _P, _P, _P]
    L.oco_gravity_monopole.restype = _I
    L.oco_ppm.argtypes = [_P, _P, _P]
    L.oco_prim.argtypes = [_P, _D, _D, _P, _P, _P]
    L.oco_prim.restype = _I
    L.oco_kt_point.argtypes = [_I, _I, _P, _P, _D, _D, _P, _P]
    L.oco_kt_point.restype = _I
    L.oco_simpson.argtypes = [_P]
    L.oco_simpson.restype = _D
    L.oco_max_threads.restype = _I
    L.oco_rhs.argtypes = [_I, _P, _P, _P, _I, _D, _D, _P, _P, _P, _I]
    L.oco_rhs.restype = _I
    L.oco_rhs_recon.argtypes = [_I, _P, _P, _P, _I, _D, _D, _I, _P, _P, _P, _I]
    L.oco_rhs_recon.restype = _I
    L.oco_rk3_step_recon.argtypes = [_I, _P, _P, _P, _I, _D, _D, _D, _D, _D, _D, _I, _P, _I, _P, _I64, _P, _P, _I]
    L.oco_rk3_step_recon.restype = _I
    L.oco_rhs_faces.argtypes = [_I, _P, _P, _P, _I, _D, _D, _P, _P, _P, _P, _I]
    L.oco_rhs_faces.restype = _I
    L.oco_rhs_faces_recon.argtypes = [_I, _P, _P, _P, _I, _D, _D, _I, _P, _P, _P, _P, _I]
    L.oco_rhs_faces_recon.restype = _I
    L.oco_amr_reflux.argtypes = [_I, _I, _P, _I, _P, _P, _I, _I, _P, _P]
    L.oco_amr_reflux.restype = _I
    L.oco_rhs_cells.argtypes = [_I, _P, _P, _P, _I, _D, _D, _P, _I, _P, _P, _I]
    L.oco_rhs_cells.restype = _I
    L.oco_dt_from_amax.argtypes = [_I, _P, _P, _D]
    L.oco_dt_from_amax.restype = _D
    L.oco_ghost_fill.argtypes = [_I, _I, _P, _I, _P, _P]
    L.oco_ghost_fill.restype = _I
    L.oco_floors.argtypes = [_I, _P, _P, _I, _D, _D, _D, _P]
    L.oco_floors.restype = _I64
    L.oco_rk_combine.argtypes = [_I, _I, _P, _P, _I, _D, _P, _P, _P]
    L.oco_rk_combine.restype = _I
    L.oco_rk3_step.argtypes = [_I, _P, _P, _P, _I, _D, _D, _D, _D, _D, _D, _I, _P, _P, _I64, _P, _P, _I]
    L.oco_rk3_step.restype = _I
    L.oco_amr_ghost_fill.argtypes = [_I, _I, _P, _I, _P, _P, _I, _I, _P]
    L.oco_amr_ghost_fill.restype = _I
    L.oco_amr_ghost_fill_order.argtypes = [_I, _I, _P, _I, _P, _P, _I, _I, _I, _P]
    L.oco_amr_ghost_fill_order.restype = _I
    L.oco_rk3_step_amr_order.argtypes = [_I, _P, _P, _P, _I, _D, _D, _D, _D, _D, _D, _P, _P, _I, _I, _I, _P, _I64, _P,
                                         _P, _I]
    L.oco_rk3_step_amr_order.restype = _I
    L.oco_rk3_step_amr.argtypes = [_I, _P, _P, _P, _I, _D, _D, _D, _D, _D, _D, _P, _P, _I, _I, _P, _I64, _P, _P, _I]
    L.oco_rk3_step_amr.restype = _I


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def max_threads() -> int:
    return int(lib().oco_max_threads())


def ppm(stencil):
    """PPM on a 5-cell stencil u_{-2..2}: returns (u at -1/2, u at +1/2)."""
    u = _f64(stencil)
    assert u.shape == (5,)
    um, up = np.zeros(1), np.zeros(1)
    lib().oco_ppm(_p(u), _p(um), _p(up))
    return float(um[0]), float(up[0])


def prim(q, gamma=5.0 / 3.0, eps1=1e-3):
    """Point primitives: returns (v[3], p, c, bad)."""
    q = _f64(q)
    v, p, c = np.zeros(3), np.zeros(1), np.zeros(1)
    bad = lib().oco_prim(_p(q), gamma, eps1, _p(v), _p(p), _p(c))
    return v, float(p[0]), float(c[0]), int(bad)


def kt_point(k, qL, qR, gamma=5.0 / 3.0, eps1=1e-3):
    """KT flux at one quadrature point: returns (F[nf], a)."""
    qL, qR = _f64(qL), _f64(qR)
    nf = qL.shape[0]
    F, a = np.zeros(nf), np.zeros(1)
    lib().oco_kt_point(int(k), nf, _p(qL), _p(qR), gamma, eps1, _p(F), _p(a))
    return F, float(a[0])


def simpson(Fq):
    """Face average of 9 point values ordered centre, 4 edge mids, 4 corners."""
    f = _f64(Fq)
    assert f.shape == (9,)
    return float(lib().oco_simpson(_p(f)))


def rhs(edge, off, dx, nf, U, gamma=5.0 / 3.0, eps1=1e-3, nthreads=0, recon=0):
    """dU/dt of all subgrids; returns (dUdt packed [s][f][E^3], amax[s], n_bad).
    recon: 0 reconstructs the conserved fields, 1 the primitive variables."""
    edge, off, dx, U = _i32(edge), _i64(off), _f64(dx), _f64(U)
    n = edge.shape[0]
    out = np.zeros(int(np.sum(nf * edge.astype(np.int64) ** 3)))
    amax = np.zeros(n)
    nb = lib().oco_rhs_recon(n, _p(edge), _p(off), _p(dx), int(nf), gamma, eps1, int(recon), _p(U), _p(out),
                             _p(amax), int(nthreads))
    if nb < 0:
        raise ValueError("oracle rhs: bad arguments")
    return out, amax, nb


def rhs_faces(edge, off, dx, nf, U, gamma=5.0 / 3.0, eps1=1e-3, nthreads=0, recon=0):
    """rhs() plus each subgrid's boundary face fluxes, [s][6][nf][E][E]
    (face 2k + side of axis k; (t2, t1) = the other two coordinates, higher
    axis first).  Uniform edge only."""
    edge, off, dx, U = _i32(edge), _i64(off), _f64(dx), _f64(U)
    n = edge.shape[0]
    E = int(edge[0])
    assert np.all(edge == E)
    out = np.zeros(int(np.sum(nf * edge.astype(np.int64) ** 3)))
    amax = np.zeros(n)
    faces = np.zeros((n, 6, nf, E, E))
    nb = lib().oco_rhs_faces_recon(n, _p(edge), _p(off), _p(dx), int(nf), gamma, eps1, int(recon), _p(U),
                                   _p(out), _p(amax), _p(faces), int(nthreads))
    if nb < 0:
        raise ValueError("oracle rhs: bad arguments")
    return out, amax, faces, nb


def amr_reflux(E, dx, nf, level, origin, n0, periodic, faces, dUdt):
    """In place: the flux correction at coarse-fine faces of dUdt (packed
    [s][f][E^3]) from the boundary face fluxes of rhs_faces."""
    dx, lev, org = _f64(dx), _i32(level), _i32(origin).reshape(-1)
    faces = np.ascontiguousarray(faces, np.float64)
    assert dUdt.dtype == np.float64 and dUdt.flags.c_contiguous
    r = lib().oco_amr_reflux(lev.shape[0], int(E), _p(dx), int(nf), _p(lev), _p(org), int(n0), int(periodic),
                             _p(faces), _p(dUdt))
    if r != 0:
        raise ValueError(f"oracle amr_reflux failed ({r})")


def rhs_cells(edge, off, dx, nf, U, samples, gamma=5.0 / 3.0, eps1=1e-3, nthreads=0):
    """dU/dt at sampled (subgrid, interior linear cell) pairs; returns [n, nf]."""
    edge, off, dx, U = _i32(edge), _i64(off), _f64(dx), _f64(U)
    smp = _i64(samples).reshape(-1, 2)
    out = np.zeros((smp.shape[0], nf))
    nb = lib().oco_rhs_cells(edge.shape[0], _p(edge), _p(off), _p(dx), int(nf), gamma, eps1, _p(U),
                             smp.shape[0], _p(smp), _p(out), int(nthreads))
    if nb < 0:
        raise ValueError("oracle rhs_cells: bad arguments")
    return out


def dt_from_amax(dx, amax, cfl=0.4):
    dx, amax = _f64(dx), _f64(amax)
    return float(lib().oco_dt_from_amax(dx.shape[0], _p(dx), _p(amax), cfl))


def ghost_fill(E, off, nf, nbr, U):
    """In-place ghost fill of U (uniform edge E) from the 26-entry neighbour table."""
    off, nbr = _i64(off), _i32(nbr)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    r = lib().oco_ghost_fill(off.shape[0], int(E), _p(off), int(nf), _p(nbr), _p(U))
    if r != 0:
        raise ValueError(f"oracle ghost_fill failed ({r})")


def floors(edge, off, nf, U, gamma=5.0 / 3.0, rho_floor=1e-12, eps2=0.1):
    edge, off = _i32(edge), _i64(off)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    return int(lib().oco_floors(edge.shape[0], _p(edge), _p(off), int(nf), gamma, rho_floor, eps2, _p(U)))


def rk_combine(stage, edge, off, nf, dt, U0, L, U):
    edge, off, U0, L = _i32(edge), _i64(off), _f64(U0), _f64(L)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    r = lib().oco_rk_combine(int(stage), edge.shape[0], _p(edge), _p(off), int(nf), float(dt), _p(U0),
                             _p(L), _p(U))
    if r != 0:
        raise ValueError("oracle rk_combine: bad stage")


def rk3_step(edge, off, dx, nf, U, bc, nbr=None, gamma=5.0 / 3.0, eps1=1e-3, eps2=0.1,
             rho_floor=1e-12, cfl=0.4, dt_cap=0.0, nthreads=0, recon=0):
    """One SSP-RK3 step in place; returns (dt, floor firings, status).
    recon: 0 reconstructs the conserved fields, 1 the primitive variables."""
    edge, off, dx = _i32(edge), _i64(off), _f64(dx)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    n = edge.shape[0]
    if nbr is None:
        nbr = np.full(26 * n, -1, np.int32)
    nbr = _i32(nbr)
    dt, fired = np.zeros(1), np.zeros(1, np.int64)
    st = lib().oco_rk3_step_recon(n, _p(edge), _p(off), _p(dx), int(nf), gamma, eps1, eps2, rho_floor, cfl,
                                  float(dt_cap), int(bc), _p(nbr), int(recon), _p(U), U.size, _p(dt), _p(fired),
                                  int(nthreads))
    return float(dt[0]), int(fired[0]), int(st)


def amr_ghost_fill(E, off, nf, level, origin, n0, periodic, U, order=0):
    """In-place ghost fill across refinement levels (same level, coarser by
    injection (order 0) or limited linear prolongation (order 1), finer by
    8-cell mean); origin is [n, 3] in cells of each level."""
    off, lev, org = _i64(off), _i32(level), _i32(origin).reshape(-1)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    if order == 0:
        r = lib().oco_amr_ghost_fill(off.shape[0], int(E), _p(off), int(nf), _p(lev), _p(org), int(n0),
                                     int(periodic), _p(U))
    else:
        r = lib().oco_amr_ghost_fill_order(off.shape[0], int(E), _p(off), int(nf), _p(lev), _p(org), int(n0),
                                           int(periodic), int(order), _p(U))
    if r != 0:
        raise ValueError(f"oracle amr_ghost_fill failed ({r})")


def rk3_step_amr(edge, off, dx, nf, U, level, origin, n0, periodic, gamma=5.0 / 3.0, eps1=1e-3, eps2=0.1,
                 rho_floor=1e-12, cfl=0.4, dt_cap=0.0, nthreads=0, order=0):
    """One SSP-RK3 step in place with the ghost fill across levels
    (prolongation order as in amr_ghost_fill)."""
    edge, off, dx = _i32(edge), _i64(off), _f64(dx)
    lev, org = _i32(level), _i32(origin).reshape(-1)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    dt, fired = np.zeros(1), np.zeros(1, np.int64)
    st = lib().oco_rk3_step_amr_order(edge.shape[0], _p(edge), _p(off), _p(dx), int(nf), gamma, eps1, eps2,
                                      rho_floor, cfl, float(dt_cap), _p(lev), _p(org), int(n0), int(periodic),
                                      int(order), _p(U), U.size, _p(dt), _p(fired), int(nthreads))
    return float(dt[0]), int(fired[0]), int(st)


def gravity_monopole(E, off, nf, nbr, dx, U, G=1.0, r_s=2.0 / 0.34):
    """Same-level monopole interactions (reading R18) of a uniform-edge batch
    with a neighbour table: returns (phi [n_sub * E^3], g [n_sub * 3 * E^3])."""
    off, nbr = _i64(off), _i32(nbr)
    assert U.dtype == np.float64 and U.flags.c_contiguous
    n = off.shape[0]
    phi = np.zeros(n * E ** 3)
    g = np.zeros(3 * n * E ** 3)
    r = lib().oco_gravity_monopole(n, int(E), _p(off), int(nf), _p(nbr), float(dx), float(G), float(r_s), _p(U),
                                   _p(phi), _p(g))
    if r != 0:
        raise ValueError("oracle gravity_monopole: bad arguments")
    return phi, g

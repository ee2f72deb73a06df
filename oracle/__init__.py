"""Plain FP64 CPU oracle of the checkerboard SU(3) heatbath sweep.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  The CUDA
library and its Python binding never touch it.

The arithmetic lives in ``su3_oracle.c`` (plain C, built without FMA
contraction).  This module compiles it with gcc on first use and wraps each
entry point with numpy in/out.  Links are in the canonical host layout
``U[L3, L2, L1, L0, 4, 3, 3, 2]`` (x0 fastest, then direction mu, row, column,
re/im), the layout of the CUDA library's ``su3_links_get/set``.

Every function here is pinned by CPU tests against facts that do not come from
the oracle itself (``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsu3_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into a shared library (gcc, -O2, no FP contraction)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile su3_oracle.c into libsu3_oracle.so."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


@contextlib.contextmanager
def use_library(path):
    """Route every wrapper of this module through another build of the oracle
    (the mutation tests plant mistakes in copies of su3_oracle.c)."""
    global _lib
    with _lock:
        saved = _lib
        _lib = _bind(ctypes.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    """Declare the argument and result types of every exported oracle function."""
    lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_u01_f64.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    lib.oracle_u01_f64.restype = ctypes.c_double
    lib.oracle_u01_f32.argtypes = [ctypes.c_uint32]
    lib.oracle_u01_f32.restype = ctypes.c_double
    lib.oracle_cold_start.argtypes = [_i32p, _f64p]
    lib.oracle_hot_start.argtypes = [_i32p, ctypes.c_uint64, ctypes.c_int, _f64p]
    lib.oracle_plaquette.argtypes = [_i32p, _f64p, ctypes.c_int]
    lib.oracle_plaquette.restype = ctypes.c_double
    lib.oracle_staple.argtypes = [_i32p, _f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _f64p]
    lib.oracle_half_sweep.argtypes = [_i32p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _u64p, ctypes.c_int]
    lib.oracle_sweep.argtypes = [_i32p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.c_int, _f64p, _u64p, _f64p, ctypes.c_int]
    lib.oracle_update_links.argtypes = [_i32p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        _i64p, ctypes.c_int64, ctypes.c_int, _f64p, _u64p, ctypes.c_int]
    lib.oracle_updated_links.argtypes = [_i32p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_int, _i64p, ctypes.c_int64, ctypes.c_int, _f64p, _f64p, _f64p,
                                         ctypes.c_int]
    lib.oracle_gauge_transform.argtypes = [_i32p, ctypes.c_uint64, _f64p]
    lib.oracle_kp_draws.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, _f64p, _u8p, ctypes.c_int,
                                     _i64p]
    lib.oracle_kp_draws.restype = ctypes.c_int64
    return lib


def _dims(L):
    L = [int(x) for x in L]
    if len(L) != 4:
        raise ValueError("need four extents")
    return (ctypes.c_int * 4)(*L)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check_links(L, U):
    shape = (L[3], L[2], L[1], L[0], 4, 3, 3, 2)
    if U.dtype != np.float64 or not U.flags.c_contiguous or U.shape != shape:
        raise ValueError("links must be float64 C-contiguous with shape %s" % (shape,))


def _rc(rc):
    if rc == -1:
        raise ValueError("oracle: invalid argument")
    if rc == -2:
        raise MemoryError("oracle: allocation failed")
    if rc != 0:
        raise RuntimeError("oracle: error %d" % rc)


def links_shape(L):
    return (L[3], L[2], L[1], L[0], 4, 3, 3, 2)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words -> four words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01_f64(a, b):
    return _load().oracle_u01_f64(int(a) & 0xFFFFFFFF, int(b) & 0xFFFFFFFF)


def u01_f32(a):
    return _load().oracle_u01_f32(int(a) & 0xFFFFFFFF)


def cold_start(L):
    U = np.empty(links_shape(L), dtype=np.float64)
    _rc(_load().oracle_cold_start(_dims(L), _ptr(U, ctypes.c_double)))
    return U


def hot_start(L, seed, f32=False):
    U = np.empty(links_shape(L), dtype=np.float64)
    _rc(_load().oracle_hot_start(_dims(L), ctypes.c_uint64(seed), int(bool(f32)), _ptr(U, ctypes.c_double)))
    return U


def plaquette(L, U, f32=False):
    _check_links(L, U)
    return float(_load().oracle_plaquette(_dims(L), _ptr(U, ctypes.c_double), int(bool(f32))))


def staple(L, U, site, mu, f32=False):
    _check_links(L, U)
    out = np.empty(18, dtype=np.float64)
    _rc(_load().oracle_staple(_dims(L), _ptr(U, ctypes.c_double), int(site), int(mu), int(bool(f32)),
                              _ptr(out, ctypes.c_double)))
    return out.reshape(3, 3, 2)


def half_sweep(L, beta, seed, t, mu, parity, U, f32=False, reverse=False, max_tries=1):
    """One checkerboard half-sweep in place; returns (accepted, proposed) SU(2) proposals.

    max_tries = 1: one-hit heatbath; > 1: repeat until accepted, at most max_tries proposals."""
    _check_links(L, U)
    st = np.zeros(2, dtype=np.uint64)
    _rc(_load().oracle_half_sweep(_dims(L), float(beta), ctypes.c_uint64(seed), ctypes.c_uint64(t), int(mu),
                                  int(parity), int(bool(f32)), int(bool(reverse)), _ptr(U, ctypes.c_double),
                                  _ptr(st, ctypes.c_uint64), int(max_tries)))
    return int(st[0]), int(st[1])


def sweep(L, beta, seed, t0, nsweeps, U, f32=False, max_tries=1):
    """nsweeps sweeps in place from sweep index t0; returns ((accepted, proposed), plaquette per sweep)."""
    _check_links(L, U)
    st = np.zeros(2, dtype=np.uint64)
    plaq = np.zeros(max(int(nsweeps), 1), dtype=np.float64)
    _rc(_load().oracle_sweep(_dims(L), float(beta), ctypes.c_uint64(seed), ctypes.c_uint64(t0), int(nsweeps),
                             int(bool(f32)), _ptr(U, ctypes.c_double), _ptr(st, ctypes.c_uint64),
                             _ptr(plaq, ctypes.c_double), int(max_tries)))
    return (int(st[0]), int(st[1])), plaq[: int(nsweeps)]


def update_links(L, beta, seed, t, mu, sites, U, f32=False, max_tries=1):
    _check_links(L, U)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    st = np.zeros(2, dtype=np.uint64)
    _rc(_load().oracle_update_links(_dims(L), float(beta), ctypes.c_uint64(seed), ctypes.c_uint64(t), int(mu),
                                    _ptr(s, ctypes.c_int64), s.size, int(bool(f32)), _ptr(U, ctypes.c_double),
                                    _ptr(st, ctypes.c_uint64), int(max_tries)))
    return int(st[0]), int(st[1])


def updated_links(L, beta, seed, t, mu, sites, U, f32=False, with_margins=False, max_tries=1):
    """Updated values of the listed links of direction mu, each from the unchanged U; shape (n, 3, 3, 2).

    With with_margins, also returns (n, 3) accept margins u3^2 - (1 - delta/2) per subgroup
    (accepted iff <= 0; NaN where the subgroup was skipped)."""
    _check_links(L, U)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((s.size, 3, 3, 2), dtype=np.float64)
    marg = np.empty((s.size, 3), dtype=np.float64)
    _rc(_load().oracle_updated_links(_dims(L), float(beta), ctypes.c_uint64(seed), ctypes.c_uint64(t), int(mu),
                                     _ptr(s, ctypes.c_int64), s.size, int(bool(f32)), _ptr(U, ctypes.c_double),
                                     _ptr(out, ctypes.c_double), _ptr(marg, ctypes.c_double), int(max_tries)))
    return (out, marg) if with_margins else out


def gauge_transform(L, seed, U):
    _check_links(L, U)
    _rc(_load().oracle_gauge_transform(_dims(L), ctypes.c_uint64(seed), _ptr(U, ctypes.c_double)))


def kp_draws(alpha, seed, n, max_tries=1, with_tries=False):
    """n Kennedy-Pendleton draws at fixed alpha with up to max_tries proposals each;
    returns (quaternions (n,4), accepted (n,) bool[, proposals drawn])."""
    out = np.zeros((int(n), 4), dtype=np.float64)
    acc = np.zeros(int(n), dtype=np.uint8)
    tries = ctypes.c_int64(0)
    _load().oracle_kp_draws(float(alpha), ctypes.c_uint64(seed), int(n), _ptr(out, ctypes.c_double),
                            _ptr(acc, ctypes.c_uint8), int(max_tries), ctypes.byref(tries))
    if with_tries:
        return out, acc.astype(bool), tries.value
    return out, acc.astype(bool)


def as_complex(U):
    """View (..., 3, 3, 2) real links as (..., 3, 3) complex128."""
    return U[..., 0] + 1j * U[..., 1]


def hot_chain(L, beta, seed, nsweeps, f32=False):
    """Hot start from `seed`, then `nsweeps` sweeps from sweep index 0.

    Returns (links, plaquette per sweep, (accepted, proposed), seconds spent in
    the sweeps).  A module-level function so that a `spawn` process pool can
    run several chains at once (each in one thread)."""
    import time
    build()
    U = hot_start(L, seed, f32=f32)
    t0 = time.perf_counter()
    stats, plaq = sweep(L, beta, seed, 0, nsweeps, U, f32=f32)
    return U, plaq, stats, time.perf_counter() - t0

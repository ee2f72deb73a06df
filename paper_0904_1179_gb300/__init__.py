"""GB300-native checkerboard SU(3) heatbath sweep (Berg & Wu, arXiv:0904.1179).

Thin ctypes binding of libsu3 (``include/su3.h``): argument marshalling only.
Every step of the sweep, the start configurations, the plaquette and the layout
conversions run in the library's sm_103a kernels.  There is no CPU fallback:
importing the binding without the built library, or calling it without a CUDA
device, raises.

The function names are those of the C ABI.  ``Lattice`` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "SU3_COLD", "SU3_HOT", "SU3_FP64", "SU3_FP32_MIXED", "SU3_FP32_EFT", "Su3Error", "load_library", "library_path",
    "su3_create", "su3_create_ex", "su3_destroy", "su3_sweep", "su3_sweep_measured", "su3_half_sweep", "su3_plaquette",
    "su3_decomp_create", "su3_decomp_plan", "su3_decomp_info",
    "su3_links_get", "su3_links_set", "su3_sweep_count", "su3_set_sweep_count", "su3_set_stats", "su3_stats",
    "su3_info", "su3_set_block_size", "su3_set_lanes", "su3_set_schedule", "su3_get_schedule", "su3_sweep_debug",
    "SU3_SCHED_AUTO", "SU3_SCHED_PHASES", "SU3_SCHED_PERSISTENT", "SU3_SCHED_PER_DIRECTION", "SU3_SCHED_CHAINED", "su3_bounds_status", "use_library", "su3_set_heatbath", "su3_batch_create", "su3_batch_sweep", "su3_batch_plaquettes",
    "su3_batch_links_get", "su3_batch_links_set", "su3_batch_size", "su3_batch_config", "su3_batch_get_config",
    "su3_batch_autotune", "su3_batch_debug", "su3_status", "Batch", "su3_plaquette_noalloc", "su3_last_error", "su3_version", "Lattice", "links_shape", "EXPORTS",
]

SU3_COLD, SU3_HOT = 0, 1
SU3_FP64, SU3_FP32_MIXED, SU3_FP32_EFT = 0, 1, 2
SU3_SCHED_AUTO, SU3_SCHED_PHASES, SU3_SCHED_PERSISTENT, SU3_SCHED_PER_DIRECTION, SU3_SCHED_CHAINED = 0, 1, 2, 3, 4
SU3_OK, SU3_EINVAL, SU3_ENOMEM, SU3_ECUDA, SU3_ETIMEOUT, SU3_ESIZE = 0, -1, -2, -3, -4, -5
_CODES = {SU3_EINVAL: "SU3_EINVAL", SU3_ENOMEM: "SU3_ENOMEM", SU3_ECUDA: "SU3_ECUDA",
          SU3_ETIMEOUT: "SU3_ETIMEOUT", SU3_ESIZE: "SU3_ESIZE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsu3.so")
_lock = threading.Lock()
_lib = None

_h = ctypes.c_void_p
_u64 = ctypes.c_uint64
_pu64 = ctypes.POINTER(ctypes.c_uint64)
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)

# (name, restype, argtypes) of every C entry point declared in include/su3.h.
EXPORTS = [
    ("su3_create", ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_double, _u64, ctypes.c_int, ctypes.POINTER(_h)]),
    ("su3_create_ex", ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_double, _u64, ctypes.c_int, ctypes.c_int,
                                                            ctypes.c_void_p, ctypes.POINTER(_h)]),
    ("su3_destroy", ctypes.c_int, [_h]),
    ("su3_sweep", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_sweep_measured", ctypes.c_int, [_h, ctypes.c_int, _pd]),
    ("su3_decomp_create", ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_double, _u64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(_h)]),
    ("su3_decomp_plan", ctypes.c_int, [ctypes.c_int] * 7 + [ctypes.POINTER(ctypes.c_int),
                                                           ctypes.POINTER(ctypes.c_longlong)]),
    ("su3_decomp_info", ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_longlong)]),
    ("su3_half_sweep", ctypes.c_int, [_h, ctypes.c_int, ctypes.c_int]),
    ("su3_plaquette", ctypes.c_double, [_h]),
    ("su3_links_get", ctypes.c_int, [_h, _pd, ctypes.c_size_t]),
    ("su3_links_set", ctypes.c_int, [_h, _pd, ctypes.c_size_t]),
    ("su3_sweep_count", ctypes.c_int, [_h, _pu64]),
    ("su3_set_sweep_count", ctypes.c_int, [_h, _u64]),
    ("su3_set_stats", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_stats", ctypes.c_int, [_h, _pu64, _pu64]),
    ("su3_info", ctypes.c_int, [_h, _pi, _pd, _pu64, _pi]),
    ("su3_set_block_size", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_set_lanes", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_set_schedule", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_get_schedule", ctypes.c_int, [_h, _pi]),
    ("su3_sweep_debug", ctypes.c_int, [_h, ctypes.c_double, ctypes.c_int]),
    ("su3_bounds_status", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), ctypes.c_int]),
    ("su3_set_heatbath", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _pd, _pu64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(_h)]),
    ("su3_batch_sweep", ctypes.c_int, [_h, ctypes.c_int]),
    ("su3_batch_plaquettes", ctypes.c_int, [_h, _pd]),
    ("su3_batch_links_get", ctypes.c_int, [_h, ctypes.c_int, _pd, ctypes.c_size_t]),
    ("su3_batch_links_set", ctypes.c_int, [_h, ctypes.c_int, _pd, ctypes.c_size_t]),
    ("su3_batch_size", ctypes.c_int, [_h, _pi]),
    ("su3_batch_config", ctypes.c_int, [_h, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("su3_batch_get_config", ctypes.c_int, [_h, _pi, _pi, _pi]),
    ("su3_batch_autotune", ctypes.c_int, [_h, _pi, _pi, _pi]),
    ("su3_batch_debug", ctypes.c_int, [_h, ctypes.c_double, ctypes.c_int]),
    ("su3_status", ctypes.c_int, [_h]),
    ("su3_plaquette_noalloc", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5 + [ctypes.c_void_p,
                                                                                      ctypes.c_void_p]),
    ("su3_last_error", ctypes.c_char_p, []),
    ("su3_version", ctypes.c_char_p, []),
]


class Su3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_CODES.get(code, str(code)), msg))
        self.code = code


def library_path() -> str:
    return _LIB_PATH


def use_library(path):
    """Use another build of the library (e.g. the bounds-checked libsu3_bounds.so) in
    this process; call before the first use of any su3_* function."""
    global _LIB_PATH
    with _lock:
        if _lib is not None and os.path.abspath(path) != os.path.abspath(_LIB_PATH):
            raise RuntimeError("libsu3 is already loaded from %s" % _LIB_PATH)
        _LIB_PATH = os.path.abspath(path)


def load_library():
    """Load libsu3.so (built by paper_0904_1179_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libsu3.so is not built (run `python -m paper_0904_1179_gb300.build` or "
                              "__graft_entry__.build()); there is no CPU fallback")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, res, args in EXPORTS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != SU3_OK:
        raise Su3Error(rc, su3_last_error())


def su3_last_error() -> str:
    return load_library().su3_last_error().decode()


def su3_version() -> str:
    return load_library().su3_version().decode()


def su3_create(L0, L1, L2, L3, beta, seed, start):
    h = _h()
    _check(load_library().su3_create(L0, L1, L2, L3, beta, seed, start, ctypes.byref(h)))
    return h


def su3_create_ex(L0, L1, L2, L3, beta, seed, start, precision, cuda_stream=None):
    """cuda_stream: a raw cudaStream_t (int), e.g. ``torch.cuda.current_stream().cuda_stream``, or None."""
    h = _h()
    _check(load_library().su3_create_ex(L0, L1, L2, L3, beta, seed, start, precision,
                                        ctypes.c_void_p(cuda_stream or None), ctypes.byref(h)))
    return h


def su3_decomp_create(L0, L1, L2, L3, beta, seed, start, precision, ndmpi, mpifactor, lbcex=1, cuda_stream=None):
    h = _h()
    _check(load_library().su3_decomp_create(L0, L1, L2, L3, beta, seed, start, precision, ndmpi, mpifactor, lbcex,
                                            ctypes.c_void_p(cuda_stream or None), ctypes.byref(h)))
    return h


def su3_decomp_plan(L, ndmpi, mpifactor, lbcex=1):
    """(number of sublattices, links copied by the exchange per sweep), computed on the host."""
    n = ctypes.c_int()
    halo = ctypes.c_longlong()
    _check(load_library().su3_decomp_plan(*[int(x) for x in L], int(ndmpi), int(mpifactor), int(lbcex),
                                          ctypes.byref(n), ctypes.byref(halo)))
    return n.value, halo.value


def su3_decomp_info(h):
    """(ndmpi, mpifactor, lbcex, number of sublattices, links copied by the exchange per sweep)."""
    v = [ctypes.c_int() for _ in range(4)]
    n = ctypes.c_longlong()
    _check(load_library().su3_decomp_info(h, *[ctypes.byref(x) for x in v], ctypes.byref(n)))
    return tuple(x.value for x in v) + (n.value,)


def su3_destroy(h):
    _check(load_library().su3_destroy(h))


def su3_sweep(h, nsweeps):
    _check(load_library().su3_sweep(h, nsweeps))


def su3_sweep_measured(h, nsweeps):
    """nsweeps sweeps with the fused plaquette; returns the plaquette after each sweep."""
    out = np.empty(max(int(nsweeps), 0), dtype=np.float64)
    _check(load_library().su3_sweep_measured(h, int(nsweeps), out.ctypes.data_as(_pd)))
    return out


def su3_half_sweep(h, mu, parity):
    _check(load_library().su3_half_sweep(h, mu, parity))


def su3_plaquette(h) -> float:
    v = load_library().su3_plaquette(h)
    if v != v:  # NaN signals failure
        raise Su3Error(SU3_ECUDA, su3_last_error())
    return v


def _host_buffer(buf, writable):
    if not isinstance(buf, np.ndarray) or buf.dtype != np.float64 or not buf.flags.c_contiguous:
        raise TypeError("links buffer must be a C-contiguous float64 numpy array")
    if writable and not buf.flags.writeable:
        raise TypeError("links buffer is read-only")
    return buf.ctypes.data_as(_pd), buf.size


def su3_links_get(h, out):
    ptr, n = _host_buffer(out, True)
    _check(load_library().su3_links_get(h, ptr, n))
    return out


def su3_links_set(h, links):
    ptr, n = _host_buffer(links, False)
    _check(load_library().su3_links_set(h, ptr, n))


def su3_sweep_count(h) -> int:
    v = ctypes.c_uint64()
    _check(load_library().su3_sweep_count(h, ctypes.byref(v)))
    return v.value


def su3_set_sweep_count(h, n):
    _check(load_library().su3_set_sweep_count(h, n))


def su3_set_stats(h, enable):
    _check(load_library().su3_set_stats(h, int(bool(enable))))


def su3_stats(h):
    a, p = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().su3_stats(h, ctypes.byref(a), ctypes.byref(p)))
    return a.value, p.value


def su3_info(h):
    dims = (ctypes.c_int * 4)()
    beta = ctypes.c_double()
    seed = ctypes.c_uint64()
    prec = ctypes.c_int()
    _check(load_library().su3_info(h, dims, ctypes.byref(beta), ctypes.byref(seed), ctypes.byref(prec)))
    return tuple(dims), beta.value, seed.value, prec.value


def su3_set_block_size(h, threads):
    _check(load_library().su3_set_block_size(h, threads))


def su3_set_lanes(h, lanes):
    """0: automatic; 1: one thread per link (or link pair); 4: four lanes per link."""
    _check(load_library().su3_set_lanes(h, int(lanes)))


def su3_set_schedule(h, schedule):
    """SU3_SCHED_AUTO, SU3_SCHED_PHASES (eight half-sweep kernels), SU3_SCHED_PERSISTENT (one kernel),
    SU3_SCHED_PER_DIRECTION (one persistent kernel per direction) or SU3_SCHED_CHAINED (eight chained
    half-sweep kernels)."""
    _check(load_library().su3_set_schedule(h, int(schedule)))


def su3_get_schedule(h):
    v = ctypes.c_int(0)
    _check(load_library().su3_get_schedule(h, ctypes.byref(v)))
    return v.value


def su3_sweep_debug(h, wait_limit_s, withhold_item=-1):
    _check(load_library().su3_sweep_debug(h, float(wait_limit_s), int(withhold_item)))


def su3_bounds_status(clear=False):
    """Bounds-checked build only: 1 if a link access was out of range since the last clear, else 0."""
    v = ctypes.c_uint(0)
    _check(load_library().su3_bounds_status(ctypes.byref(v), int(bool(clear))))
    return v.value


def su3_set_heatbath(h, max_tries):
    """1: one-hit heatbath (default); > 1: repeat until accepted, at most max_tries proposals."""
    _check(load_library().su3_set_heatbath(h, int(max_tries)))


def su3_batch_create(dims, betas, seeds, start, precision, cuda_stream=None):
    """dims: sequence of n (L0, L1, L2, L3); betas, seeds: length n."""
    n = len(dims)
    if len(betas) != n or len(seeds) != n:
        raise ValueError("dims, betas and seeds must have the same length")
    d = (ctypes.c_int * (4 * n))(*[int(x) for L in dims for x in L])
    b = (ctypes.c_double * n)(*[float(x) for x in betas])
    s = (ctypes.c_uint64 * n)(*[int(x) for x in seeds])
    h = _h()
    _check(load_library().su3_batch_create(n, d, b, s, int(start), int(precision), ctypes.c_void_p(cuda_stream or None),
                                           ctypes.byref(h)))
    return h


def su3_batch_sweep(h, nsweeps):
    _check(load_library().su3_batch_sweep(h, nsweeps))


def su3_batch_plaquettes(h, n):
    out = (ctypes.c_double * n)()
    _check(load_library().su3_batch_plaquettes(h, out))
    return list(out)


def su3_batch_links_get(h, replica, out):
    ptr, n = _host_buffer(out, True)
    _check(load_library().su3_batch_links_get(h, int(replica), ptr, n))
    return out


def su3_batch_links_set(h, replica, links):
    ptr, n = _host_buffer(links, False)
    _check(load_library().su3_batch_links_set(h, int(replica), ptr, n))


def su3_batch_size(h):
    n = ctypes.c_int()
    _check(load_library().su3_batch_size(h, ctypes.byref(n)))
    return n.value


def su3_batch_config(h, threads=0, blocks_per_sm=0, window=0):
    _check(load_library().su3_batch_config(h, int(threads), int(blocks_per_sm), int(window)))


def su3_batch_get_config(h):
    t, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().su3_batch_get_config(h, ctypes.byref(t), ctypes.byref(b), ctypes.byref(w)))
    return t.value, b.value, w.value


def su3_batch_autotune(h):
    t, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().su3_batch_autotune(h, ctypes.byref(t), ctypes.byref(b), ctypes.byref(w)))
    return t.value, b.value, w.value


def su3_batch_debug(h, wait_limit_s, withhold_item=-1):
    _check(load_library().su3_batch_debug(h, float(wait_limit_s), int(withhold_item)))


def su3_status(h):
    """Synchronise; raises Su3Error (code SU3_ETIMEOUT or SU3_ECUDA) on an asynchronous failure."""
    _check(load_library().su3_status(h))


def su3_plaquette_noalloc(links_ptr, dims, precision, out_ptr, cuda_stream=None):
    """Mean plaquette of a device-resident link store (library device layout) into the
    device double at out_ptr, without any allocation; asynchronous on cuda_stream.

    For callers that cannot allocate device memory (stream capture, pool-only
    runtimes).  Pointers are raw device addresses (ints), e.g. tensor.data_ptr()."""
    L0, L1, L2, L3 = (int(x) for x in dims)
    _check(load_library().su3_plaquette_noalloc(ctypes.c_void_p(links_ptr), L0, L1, L2, L3, int(precision),
                                                ctypes.c_void_p(out_ptr), ctypes.c_void_p(cuda_stream or None)))


def links_shape(L):
    """Canonical host layout of a configuration: U[L3][L2][L1][L0][mu][row][col][re/im]."""
    return (L[3], L[2], L[1], L[0], 4, 3, 3, 2)


class Batch:
    """Owning wrapper of a batch handle: n replicas swept together (four chained launches per sweep)."""

    def __init__(self, dims, betas, seeds, start=SU3_HOT, precision=SU3_FP32_MIXED, stream=None):
        self.dims = [tuple(int(x) for x in L) for L in dims]
        self.n = len(self.dims)
        self.handle = su3_batch_create(self.dims, betas, seeds, start, precision, stream)
        self.precision = int(precision)

    def close(self):
        if self.handle is not None:
            su3_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def updates_per_sweep(self):
        return int(sum(4 * np.prod(L) for L in self.dims))

    def sweep(self, n=1):
        su3_batch_sweep(self.handle, n)

    def plaquettes(self):
        return su3_batch_plaquettes(self.handle, self.n)

    def get_links(self, replica, out=None):
        if out is None:
            out = np.empty(links_shape(self.dims[replica]), dtype=np.float64)
        return su3_batch_links_get(self.handle, replica, out)

    def set_links(self, replica, links):
        su3_batch_links_set(self.handle, replica, np.ascontiguousarray(links, dtype=np.float64))

    @property
    def sweep_count(self):
        return su3_sweep_count(self.handle)

    @sweep_count.setter
    def sweep_count(self, n):
        su3_set_sweep_count(self.handle, int(n))

    def config(self, threads=0, blocks_per_sm=0, window=0):
        su3_batch_config(self.handle, threads, blocks_per_sm, window)

    def get_config(self):
        return su3_batch_get_config(self.handle)

    def autotune(self):
        return su3_batch_autotune(self.handle)

    def set_heatbath(self, max_tries):
        su3_set_heatbath(self.handle, max_tries)

    def debug(self, wait_limit_s, withhold_item=-1):
        su3_batch_debug(self.handle, wait_limit_s, withhold_item)

    def status(self):
        su3_status(self.handle)


class Lattice:
    """Owning wrapper of one su3 handle."""

    def __init__(self, dims, beta, seed, start=SU3_HOT, precision=SU3_FP64, stream=None, decomp=None):
        """decomp = (ndmpi, mpifactor, lbcex): the domain decomposition emulated on one device."""
        self.dims = tuple(int(x) for x in dims)
        if decomp is None:
            self.handle = su3_create_ex(*self.dims, float(beta), int(seed), int(start), int(precision), stream)
        else:
            nd, nf, ex = (tuple(decomp) + (1,))[:3]
            self.handle = su3_decomp_create(*self.dims, float(beta), int(seed), int(start), int(precision), int(nd),
                                            int(nf), int(ex), stream)
        self.beta = float(beta)
        self.seed = int(seed)
        self.precision = int(precision)

    def close(self):
        if self.handle is not None:
            su3_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def volume(self):
        return int(np.prod(self.dims))

    def sweep(self, n=1):
        su3_sweep(self.handle, n)

    def decomp_info(self):
        return su3_decomp_info(self.handle)

    def sweep_measured(self, n):
        return su3_sweep_measured(self.handle, n)

    def half_sweep(self, mu, parity):
        su3_half_sweep(self.handle, mu, parity)

    def plaquette(self):
        return su3_plaquette(self.handle)

    def get_links(self, out=None):
        if out is None:
            out = np.empty(links_shape(self.dims), dtype=np.float64)
        return su3_links_get(self.handle, out)

    def set_links(self, links):
        su3_links_set(self.handle, np.ascontiguousarray(links, dtype=np.float64))

    @property
    def sweep_count(self):
        return su3_sweep_count(self.handle)

    @sweep_count.setter
    def sweep_count(self, n):
        su3_set_sweep_count(self.handle, int(n))

    def set_stats(self, enable=True):
        su3_set_stats(self.handle, enable)

    def stats(self):
        return su3_stats(self.handle)

    def set_block_size(self, threads):
        su3_set_block_size(self.handle, threads)

    def set_lanes(self, lanes):
        su3_set_lanes(self.handle, lanes)

    def set_schedule(self, schedule):
        su3_set_schedule(self.handle, schedule)

    @property
    def schedule(self):
        return su3_get_schedule(self.handle)

    def debug(self, wait_limit_s, withhold_item=-1):
        su3_sweep_debug(self.handle, wait_limit_s, withhold_item)

    def status(self):
        su3_status(self.handle)

    def set_heatbath(self, max_tries):
        su3_set_heatbath(self.handle, max_tries)

"""Thin ctypes binding of libnd (include/nd.h): argument marshalling only.

Every step of the computation runs in the CUDA library.  There is no CPU
fallback: if the library is missing or cannot be loaded this module raises.

Arrays may be numpy arrays (host memory; on_device = 0) or CUDA torch tensors
(device memory; on_device = 1).  Results come back in the same kind of
memory as the input graph: numpy for a host graph, torch CUDA tensors for a
device graph.  Calls run on torch's current CUDA stream unless a stream is
given.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

ND_OK, ND_E_INVAL, ND_E_UNSUPPORTED_RS, ND_E_NOMEM, ND_E_CUDA, ND_E_NOT_CONVERGED, \
    ND_E_TIMEOUT, ND_E_TOO_LARGE, ND_E_BUSY = range(9)
ND_SND, ND_AND, ND_AND_NN = 0, 1, 2
MODES = {"snd": ND_SND, "and": ND_AND, "and_nn": ND_AND_NN}

# every function include/nd.h declares (tests/test_abi.py checks the two lists agree)
SYMBOLS = [
    "nd_normalize", "nd_build_incidence", "nd_build_incidence_ex", "nd_build_incidence_batch",
    "nd_incidence_info", "nd_incidence_bytes", "nd_r_cliques", "nd_s_degree",
    "nd_snd", "nd_and", "nd_iterate_k", "nd_and_partial", "nd_and_until",
    "nd_truss_classic", "nd_count_equal", "nd_kendall_tau_b",
    "nd_prof_enable", "nd_prof_read", "nd_last_passes", "nd_autotune",
    "nd_core_snd_noalloc", "nd_set_wait_limit", "nd_set_handle_memory_limit",
    "nd_free", "nd_strerror", "nd_last_error", "nd_abi_version",
]

_lock = threading.Lock()
_lib = None


class NDError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("on_device", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnd (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and (not os.path.exists(path) or _build._stale()):
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libnd is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        i32, i64, vp, ci = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        P = ctypes.POINTER
        lib.nd_build_incidence.argtypes = [P(_CSR), ci, ci, vp, P(vp)]
        lib.nd_build_incidence_ex.argtypes = [P(_CSR), ci, ci, ctypes.c_uint, vp, P(vp)]
        lib.nd_build_incidence_batch.argtypes = [P(_CSR), ci, ci, ci, vp, P(vp), vp]
        lib.nd_incidence_info.argtypes = [vp, P(i64), P(i64), P(ci)]
        lib.nd_r_cliques.argtypes = [vp, vp, ci, vp]
        lib.nd_s_degree.argtypes = [vp, vp, ci, vp]
        lib.nd_snd.argtypes = [vp, vp, ci, i32, P(i32), vp]
        lib.nd_and.argtypes = [vp, vp, ci, ci, i32, P(i32), P(i64), vp]
        lib.nd_iterate_k.argtypes = [vp, ci, i32, vp, ci, ci, P(i32), vp]
        lib.nd_truss_classic.argtypes = [vp, i64, vp, ci, vp]
        lib.nd_prof_enable.argtypes = [ci]
        lib.nd_prof_read.argtypes = [ci, P(ctypes.c_char_p), P(i64), P(ctypes.c_double)]
        lib.nd_last_passes.argtypes = [vp, vp, vp, vp, i32, P(i32)]
        lib.nd_autotune.argtypes = [vp, i32, vp, vp, P(ctypes.c_double)]
        lib.nd_and_partial.argtypes = [vp, vp, i64, ci, vp, i32, P(i32), P(i64), vp]
        lib.nd_and_until.argtypes = [vp, ctypes.c_double, vp, ci, i32, P(i32), P(i64), P(ci), vp]
        lib.nd_count_equal.argtypes = [vp, vp, i64, ci, P(i64), vp]
        lib.nd_kendall_tau_b.argtypes = [vp, vp, i64, ci, P(ctypes.c_double), vp, vp]
        lib.nd_incidence_bytes.argtypes = [vp, P(i64)]
        lib.nd_core_snd_noalloc.argtypes = [vp, vp, i64, i64, vp, i32, P(i32), vp]
        lib.nd_normalize.argtypes = [vp, vp, i64, i64, ci, vp, vp, i64, P(i64), vp]
        lib.nd_set_wait_limit.argtypes = [ctypes.c_double]
        lib.nd_set_handle_memory_limit.argtypes = [i64]
        lib.nd_free.argtypes = [vp]
        lib.nd_free.restype = None
        lib.nd_strerror.argtypes = [ci]
        lib.nd_strerror.restype = ctypes.c_char_p
        lib.nd_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS:
            f = getattr(lib, name)
            if f.restype is ctypes.c_int:  # default restype: nd_status
                f.restype = ci
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != ND_OK:
        lib = load()
        raise NDError(st, where, f"{lib.nd_strerror(st).decode()}: {lib.nd_last_error().decode()}")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_ptr(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _ptr(x):
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _empty(n, like_device: bool, device=None, dtype="int32"):
    if like_device:
        import torch
        return torch.empty(n, dtype=getattr(torch, dtype), device=device)
    return np.empty(n, dtype=dtype)


class Incidence:
    """A built r-clique -> s-clique incidence (library-owned device memory)."""

    def __init__(self, handle, r, s, on_device, device, stream):
        self._h = handle
        self.r, self.s = r, s
        self.on_device = on_device
        self.device = device
        self._stream = stream
        n_r, n_inc, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(load().nd_incidence_info(self._h, ctypes.byref(n_r), ctypes.byref(n_inc),
                                        ctypes.byref(q)), "nd_incidence_info")
        self.num_r, self.num_incidences, self.q = n_r.value, n_inc.value, q.value

    # -- lifetime
    def free(self):
        if self._h is not None and self._h.value:
            load().nd_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _alloc(self, n, dtype="int32"):
        return _empty(n, self.on_device, self.device, dtype)

    def _sp(self, stream):
        return _stream_ptr(stream if stream is not None else self._stream)

    # -- calls (same names as the C ABI)
    def incidence_info(self):
        return self.num_r, self.num_incidences, self.q

    def incidence_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(load().nd_incidence_bytes(self._h, ctypes.byref(b)), "nd_incidence_bytes")
        return b.value

    def r_cliques(self, stream=None):
        out = self._alloc(self.num_r * self.r)
        _check(load().nd_r_cliques(self._h, _ptr(out), int(self.on_device), self._sp(stream)),
               "nd_r_cliques")
        return out.reshape(self.num_r, self.r)

    def s_degree(self, stream=None):
        out = self._alloc(self.num_r)
        _check(load().nd_s_degree(self._h, _ptr(out), int(self.on_device), self._sp(stream)),
               "nd_s_degree")
        return out

    def snd(self, max_iters: int = 1 << 30, out=None, stream=None):
        """SND (Alg. 2) to convergence.  Returns (tau, updating passes)."""
        tau = self._alloc(self.num_r) if out is None else out
        it = ctypes.c_int32()
        _check(load().nd_snd(self._h, _ptr(tau), int(self.on_device), int(max_iters),
                             ctypes.byref(it), self._sp(stream)), "nd_snd")
        return tau, it.value

    def and_(self, notify: bool = True, max_iters: int = 1 << 30, out=None, stream=None):
        """AND (Alg. 3) to convergence.  Returns (tau, updating passes, evaluations)."""
        tau = self._alloc(self.num_r) if out is None else out
        it, ev = ctypes.c_int32(), ctypes.c_int64()
        _check(load().nd_and(self._h, _ptr(tau), int(self.on_device), int(bool(notify)),
                             int(max_iters), ctypes.byref(it), ctypes.byref(ev), self._sp(stream)),
               "nd_and")
        return tau, it.value, ev.value

    def and_partial(self, members, max_iters: int = 1 << 30, out=None, stream=None):
        """PartialAnd on the r-clique ids `members` (numpy uint32 for a host
        graph, CUDA int32/uint32 tensor for a device graph).
        Returns (tau, updating passes, evaluations)."""
        if _is_torch(members):
            ids = members.to(__import__("torch").int32).contiguous()
        else:
            ids = np.ascontiguousarray(np.asarray(members, dtype=np.uint32))
        tau = self._alloc(self.num_r) if out is None else out
        it, ev = ctypes.c_int32(), ctypes.c_int64()
        _check(load().nd_and_partial(self._h, _ptr(ids), len(ids), int(_is_torch(ids)), _ptr(tau),
                                     int(max_iters), ctypes.byref(it), ctypes.byref(ev), self._sp(stream)),
               "nd_and_partial")
        return tau, it.value, ev.value

    def and_until(self, active_ratio: float, max_iters: int = 1 << 30, out=None, stream=None):
        """AND with the active-ratio stopping rule.  Returns (tau, passes, evaluations, stopped)."""
        tau = self._alloc(self.num_r) if out is None else out
        it, ev, stop = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int()
        _check(load().nd_and_until(self._h, float(active_ratio), _ptr(tau), int(self.on_device), int(max_iters),
                                   ctypes.byref(it), ctypes.byref(ev), ctypes.byref(stop), self._sp(stream)),
               "nd_and_until")
        return tau, it.value, ev.value, bool(stop.value)

    def iterate_k(self, mode: str, k: int, tau=None, stream=None):
        """At most k passes of mode ('snd', 'and', 'and_nn') from tau (or d_s).
        Returns (tau, updating passes); tau is a new array."""
        if tau is None:
            buf = self._alloc(self.num_r)
            given = 0
        else:
            if _is_torch(tau) != bool(self.on_device):
                raise ValueError("tau must live where the graph lives")
            buf = tau.clone() if _is_torch(tau) else np.array(tau, dtype=np.int32, copy=True)
            given = 1
        up = ctypes.c_int32()
        _check(load().nd_iterate_k(self._h, MODES[mode], int(k), _ptr(buf), given,
                                   int(self.on_device), ctypes.byref(up), self._sp(stream)),
               "nd_iterate_k")
        return buf, up.value

    def autotune(self, passes: int = 2, stream=None):
        """nd_autotune: pick the fastest bucket thresholds for this handle (and
        cache them for later builds of the same size class).
        Returns ((t0, t1, t2), ms of `passes` SND passes with them)."""
        thr = np.zeros(3, np.int32)
        ms = ctypes.c_double()
        _check(load().nd_autotune(self._h, int(passes), self._sp(stream), _ptr(thr), ctypes.byref(ms)),
               "nd_autotune")
        return tuple(int(x) for x in thr), ms.value

    def last_passes(self, with_incidences: bool = False):
        """(changed, evaluated[, incidences]) per pass of the last iteration call."""
        lib = load()
        n = ctypes.c_int32()
        _check(lib.nd_last_passes(self._h, None, None, None, 0, ctypes.byref(n)), "nd_last_passes")
        ch = np.zeros(max(n.value, 1), np.int64)
        ev = np.zeros(max(n.value, 1), np.int64)
        inc = np.zeros(max(n.value, 1), np.int64)
        _check(lib.nd_last_passes(self._h, _ptr(ch), _ptr(ev), _ptr(inc), n.value, ctypes.byref(n)),
               "nd_last_passes")
        if with_incidences:
            return ch[:n.value], ev[:n.value], inc[:n.value]
        return ch[:n.value], ev[:n.value]


ND_BUILD_ON_THE_FLY = 1


def build_incidence(row_ptr, col, r: int, s: int, stream=None, on_the_fly: bool = False) -> Incidence:
    """nd_build_incidence on a CSR given as numpy arrays (host) or CUDA tensors.
    on_the_fly: store no incidence and find the s-cliques again on every pass
    (nd_build_incidence_ex with ND_BUILD_ON_THE_FLY; (1,2) and (2,3))."""
    lib = load()
    on_device = _is_torch(row_ptr)
    if on_device != _is_torch(col):
        raise ValueError("row_ptr and col must both be host arrays or both CUDA tensors")
    device = None
    if on_device:
        import torch
        if not (row_ptr.is_cuda and col.is_cuda):
            raise ValueError("torch tensors must be on a CUDA device")
        row_ptr = row_ptr.to(torch.int64).contiguous()
        col = col.to(torch.int32).contiguous()
        device = row_ptr.device
        n, nnz = row_ptr.numel() - 1, col.numel()
    else:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n, nnz = row_ptr.size - 1, col.size
    csr = _CSR(n, nnz, _ptr(row_ptr).value, _ptr(col).value if nnz else None, int(on_device))
    h = ctypes.c_void_p()
    if on_the_fly:
        _check(lib.nd_build_incidence_ex(ctypes.byref(csr), int(r), int(s), ND_BUILD_ON_THE_FLY,
                                         _stream_ptr(stream), ctypes.byref(h)), "nd_build_incidence_ex")
    else:
        _check(lib.nd_build_incidence(ctypes.byref(csr), int(r), int(s), _stream_ptr(stream),
                                      ctypes.byref(h)), "nd_build_incidence")
    return Incidence(h, r, s, on_device, device, stream)


def build_incidence_batch(graphs, r: int, s: int, stream=None):
    """nd_build_incidence_batch on a list of (row_ptr, col) pairs, all numpy or
    all CUDA tensors.  Returns (Incidence of the disjoint union, r_offsets):
    graph i's results are the slice [r_offsets[i], r_offsets[i+1])."""
    lib = load()
    count = len(graphs)
    arr = (_CSR * max(count, 1))()
    keep = []
    on_device = None
    device = None
    for i, (rp, col) in enumerate(graphs):
        dev = _is_torch(rp)
        if on_device is None:
            on_device = dev
        if dev != on_device or dev != _is_torch(col):
            raise ValueError("all graphs must be host arrays or all CUDA tensors")
        if dev:
            import torch
            rp = rp.to(torch.int64).contiguous()
            col = col.to(torch.int32).contiguous()
            device = rp.device
            n, nnz = rp.numel() - 1, col.numel()
        else:
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            n, nnz = rp.size - 1, col.size
        keep.append((rp, col))
        arr[i] = _CSR(n, nnz, _ptr(rp).value, _ptr(col).value if nnz else None, int(dev))
    offs = np.zeros(count + 1, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib.nd_build_incidence_batch(arr, count, int(r), int(s), _stream_ptr(stream), ctypes.byref(h),
                                        _ptr(offs)), "nd_build_incidence_batch")
    return Incidence(h, r, s, bool(on_device), device, stream), offs


def normalize(src, dst, n: int, stream=None):
    """nd_normalize: the simple undirected CSR (Section 2) of an arbitrary
    list of vertex pairs -- self-loops dropped, every pair symmetrised,
    repeats removed, rows sorted.  src, dst: int64 numpy arrays (host) or
    CUDA tensors.  Returns (row_ptr int64[n+1], col int32[nnz]) in the same
    kind of memory."""
    on_device = _is_torch(src)
    if on_device != _is_torch(dst):
        raise ValueError("src and dst must both be host arrays or both CUDA tensors")
    if on_device:
        import torch
        src = src.to(torch.int64).contiguous()
        dst = dst.to(torch.int64).contiguous()
        m = src.numel()
    else:
        src = np.ascontiguousarray(src, dtype=np.int64).ravel()
        dst = np.ascontiguousarray(dst, dtype=np.int64).ravel()
        m = src.size
    if (dst.numel() if on_device else dst.size) != m:
        raise ValueError("src and dst differ in length")
    rp = _empty(int(n) + 1, on_device, src.device if on_device else None, "int64")
    col = _empty(max(2 * m, 1), on_device, src.device if on_device else None, "int32")
    nnz = ctypes.c_int64()
    _check(load().nd_normalize(_ptr(src) if m else None, _ptr(dst) if m else None, m, int(n), int(on_device),
                               _ptr(rp), _ptr(col), 2 * m, ctypes.byref(nnz), _stream_ptr(stream)),
           "nd_normalize")
    return rp, col[:nnz.value]


def set_wait_limit(seconds: float):
    """nd_set_wait_limit: limit of every host-side wait of the library."""
    _check(load().nd_set_wait_limit(float(seconds)), "nd_set_wait_limit")


def set_handle_memory_limit(nbytes: int):
    """nd_set_handle_memory_limit: device bytes one handle may hold (0 = no limit)."""
    _check(load().nd_set_handle_memory_limit(int(nbytes)), "nd_set_handle_memory_limit")


def core_snd_noalloc(row_ptr, col, out=None, max_iters: int = 1 << 30, stream=None):
    """nd_core_snd_noalloc: core numbers from a device CSR (CUDA int64 row_ptr,
    int32 col) with no allocation inside the library; `out` (CUDA int32, n)
    is allocated here by torch if not given.  Returns (core, passes)."""
    import torch
    n = row_ptr.numel() - 1
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    it = ctypes.c_int32()
    _check(load().nd_core_snd_noalloc(_ptr(row_ptr), _ptr(col), n, col.numel(), _ptr(out),
                                      int(max_iters), ctypes.byref(it), _stream_ptr(stream)),
           "nd_core_snd_noalloc")
    return out, it.value


def truss_classic(kappa3, stream=None):
    """Classic (k-2 convention) truss numbers: kappa_3 + 2 (nd_truss_classic)."""
    on_device = _is_torch(kappa3)
    out = _empty(len(kappa3), on_device, kappa3.device if on_device else None)
    src = kappa3 if on_device else np.ascontiguousarray(kappa3, dtype=np.int32)
    _check(load().nd_truss_classic(_ptr(src), len(kappa3), _ptr(out), int(on_device),
                                   _stream_ptr(stream)), "nd_truss_classic")
    return out


def count_equal(a, b, stream=None) -> int:
    """nd_count_equal: positions where a == b (both numpy or both CUDA tensors)."""
    on_device = _is_torch(a)
    if not on_device:
        a = np.ascontiguousarray(a, dtype=np.int32)
        b = np.ascontiguousarray(b, dtype=np.int32)
    out = ctypes.c_int64()
    _check(load().nd_count_equal(_ptr(a), _ptr(b), len(a), int(on_device), ctypes.byref(out), _stream_ptr(stream)),
           "nd_count_equal")
    return out.value


def kendall_tau_b(x, y, stream=None, with_counts: bool = False):
    """nd_kendall_tau_b: Kendall's tau-b of x against y (both numpy or both
    CUDA tensors), e.g. an early-stopped tau against kappa.  With
    with_counts, also (S, ties_x, ties_y)."""
    on_device = _is_torch(x)
    if not on_device:
        x = np.ascontiguousarray(x, dtype=np.int32)
        y = np.ascontiguousarray(y, dtype=np.int32)
    if len(x) != len(y):
        raise ValueError("sequences differ in length")
    tau = ctypes.c_double()
    counts = np.zeros(3, np.int64)
    _check(load().nd_kendall_tau_b(_ptr(x), _ptr(y), len(x), int(on_device), ctypes.byref(tau), _ptr(counts),
                                   _stream_ptr(stream)), "nd_kendall_tau_b")
    if with_counts:
        return tau.value, int(counts[0]), int(counts[1]), int(counts[2])
    return tau.value


def prof_enable(on: bool = True):
    _check(load().nd_prof_enable(int(on)), "nd_prof_enable")


def prof_read() -> dict:
    """{kernel name: (launches, total ms)} recorded since prof_enable(True)."""
    lib = load()
    out = {}
    i = 0
    while True:
        name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
        if lib.nd_prof_read(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)) != ND_OK:
            break
        out[name.value.decode()] = (n.value, ms.value)
        i += 1
    return out


def strerror(status: int) -> str:
    return load().nd_strerror(int(status)).decode()


def abi_version() -> int:
    return int(load().nd_abi_version())

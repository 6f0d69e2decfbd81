"""CPU oracle for local nucleus decomposition -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it never imports them.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, compiled here
with gcc); this module only marshals numpy arrays through ctypes.
``snd_mt.c`` is the same SND (Alg. 2, Def. 4, Def. 3 by sorting) with its
loops split over OpenMP threads, used to time the CPU baseline on all host
cores; a CPU test pins it pass by pass against the single-threaded one.  The
brute-force search of Lemma 1 is written in Python because it only runs on
graphs with a handful of r-cliques.

Sections cited: Def. 1 (r-/s-cliques, S-degree), Def. 2 (kappa_s), Lemma 1,
Def. 3 (h-index), Def. 4 (update operator), Alg. 1 (peeling), Alg. 2 (SND),
Alg. 3 (AND) with the notification of Section 4.3, Def. 5 (degree levels).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_MT_PATH = os.path.join(_LIBDIR, "liboracle_mt.so")
_MT_SRC = os.path.join(_HERE, "snd_mt.c")
_lock = threading.Lock()
_lib = None
_mt = None

ERRORS = {0: "ok", -1: "invalid input", -2: "out of memory",
          -3: "an update raised tau (Thm. 1 violated)", -4: "unsupported (r,s)"}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library with gcc (plain -O2), and
    snd_mt.c into a second one with OpenMP (without it, if the compiler has
    none: the routine then runs on one thread and says so)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    if force or not os.path.exists(_MT_PATH) or os.path.getmtime(_MT_PATH) < os.path.getmtime(_MT_SRC):
        tmp = _MT_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _MT_SRC]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _MT_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.orc_create.argtypes = [i64, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(vp)]
        lib.orc_create.restype = ctypes.c_int
        lib.orc_free.argtypes = [vp]
        lib.orc_num_r.argtypes = [vp]
        lib.orc_num_r.restype = i64
        lib.orc_num_s_incidences.argtypes = [vp]
        lib.orc_num_s_incidences.restype = i64
        lib.orc_q.argtypes = [vp]
        lib.orc_r_tuples.argtypes = [vp, vp]
        lib.orc_s_degree.argtypes = [vp, vp]
        lib.orc_hindex.argtypes = [vp, i64]
        lib.orc_hindex.restype = i32
        lib.orc_peel.argtypes = [vp, vp]
        lib.orc_snd.argtypes = [vp, vp, ctypes.c_int, i32, vp, vp, vp]
        lib.orc_and.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, i32, vp, vp, vp]
        lib.orc_and_partial.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, i32, vp, vp, vp]
        lib.orc_snd_partial.argtypes = [vp, vp, ctypes.c_int, vp, i32, vp]
        lib.orc_degree_levels.argtypes = [vp, vp]
        lib.orc_kendall_tau_b.argtypes = [vp, vp, i64, vp, vp, vp]
        lib.orc_kendall_tau_b.restype = ctypes.c_double
        lib.orc_degree_levels.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int):
    if st != 0:
        raise RuntimeError(f"oracle: {ERRORS.get(st, st)}")


def hindex(values) -> int:
    """H(K), Def. 3: the largest h with at least h members of K that are >= h."""
    a = np.ascontiguousarray(np.asarray(values, dtype=np.int32).copy())
    return int(_load().orc_hindex(_ptr(a), a.size))


class Graph:
    """One graph and one (r, s) job, with the oracle's own enumeration.

    ``row_ptr`` / ``col`` must be a simple, symmetric, sorted CSR.  With
    ``incidence=True`` the oracle also lists, for every r-clique, the other
    r-cliques of each s-clique that contains it (needed by SND and AND).
    """

    def __init__(self, row_ptr, col, r: int, s: int, incidence: bool = True):
        lib = _load()
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.n = self.row_ptr.size - 1
        self.r, self.s = r, s
        if self.row_ptr.size == 0 or int(self.row_ptr[-1]) != self.col.size:
            # the C side cannot see the length of col: its offsets must end there
            raise RuntimeError("oracle: invalid input (row_ptr must end at len(col))")
        h = ctypes.c_void_p()
        _check(lib.orc_create(self.n, _ptr(self.row_ptr), _ptr(self.col), r, s, int(incidence),
                              ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.num_r = int(lib.orc_num_r(h))
        self.q = int(lib.orc_q(h))
        self.has_incidence = incidence

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    @property
    def num_incidences(self) -> int:
        return int(self._lib.orc_num_s_incidences(self._h))

    def r_cliques(self) -> np.ndarray:
        """Vertex tuples of the r-cliques in canonical (lexicographic) order."""
        out = np.zeros((self.num_r, self.r), dtype=np.int32)
        self._lib.orc_r_tuples(self._h, _ptr(out))
        return out

    def s_degree(self) -> np.ndarray:
        """d_s(R), Def. 1, counted directly from the adjacency."""
        out = np.zeros(self.num_r, dtype=np.int32)
        _check(self._lib.orc_s_degree(self._h, _ptr(out)))
        return out

    def peel(self) -> np.ndarray:
        """kappa_s by peeling, Alg. 1 (Batagelj-Zaversnik bins)."""
        out = np.zeros(self.num_r, dtype=np.int32)
        _check(self._lib.orc_peel(self._h, _ptr(out)))
        return out

    def snd(self, tau=None, max_sweeps: int = 1 << 30):
        """SND, Alg. 2.  Starts from d_s (or from ``tau``) and runs until a pass
        changes nothing or ``max_sweeps`` passes ran.

        Returns (tau, sweeps, updating_sweeps, evaluations)."""
        if not self.has_incidence:
            raise RuntimeError("build the Graph with incidence=True")
        t = np.zeros(self.num_r, dtype=np.int32) if tau is None else \
            np.ascontiguousarray(np.asarray(tau, dtype=np.int32).copy())
        sw, up, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.orc_snd(self._h, _ptr(t), int(tau is None), max_sweeps,
                                 ctypes.byref(sw), ctypes.byref(up), ctypes.byref(ev)))
        return t, sw.value, up.value, ev.value

    def and_(self, notify: bool = True, order=None, tau=None, max_sweeps: int = 1 << 30):
        """AND, Alg. 3, processed sequentially in ``order`` (default: id order).

        Returns (tau, sweeps, updating_sweeps, evaluations)."""
        if not self.has_incidence:
            raise RuntimeError("build the Graph with incidence=True")
        t = np.zeros(self.num_r, dtype=np.int32) if tau is None else \
            np.ascontiguousarray(np.asarray(tau, dtype=np.int32).copy())
        o = None
        if order is not None:
            o = np.ascontiguousarray(np.asarray(order, dtype=np.int64))
            if sorted(o.tolist()) != list(range(self.num_r)):
                raise ValueError("order must be a permutation of the r-clique ids")
        sw, up, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.orc_and(self._h, _ptr(t), int(tau is None),
                                 None if o is None else _ptr(o), int(notify), max_sweeps,
                                 ctypes.byref(sw), ctypes.byref(up), ctypes.byref(ev)))
        return t, sw.value, up.value, ev.value

    def partial_and(self, members, notify: bool = True, order=None, max_sweeps: int = 1 << 30):
        """PartialAnd (end of Section 4.3): AND restricted to the member set P
        (a boolean mask over r-cliques).  Returns (tau, sweeps, updating, evaluations)."""
        m = np.ascontiguousarray(np.asarray(members, dtype=bool).astype(np.int8))
        if m.size != self.num_r:
            raise ValueError("members must be a mask over the r-cliques")
        t = np.zeros(self.num_r, dtype=np.int32)
        o = None if order is None else np.ascontiguousarray(np.asarray(order, dtype=np.int64))
        sw, up, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.orc_and_partial(self._h, _ptr(t), 1, None if o is None else _ptr(o), int(notify),
                                         _ptr(m), max_sweeps, ctypes.byref(sw), ctypes.byref(up),
                                         ctypes.byref(ev)))
        return t, sw.value, up.value, ev.value

    def partial_snd(self, members, max_sweeps: int = 1 << 30):
        """SND restricted to the member set (synchronous counterpart used as a pin)."""
        m = np.ascontiguousarray(np.asarray(members, dtype=bool).astype(np.int8))
        t = np.zeros(self.num_r, dtype=np.int32)
        sw = ctypes.c_int32()
        _check(self._lib.orc_snd_partial(self._h, _ptr(t), 1, _ptr(m), max_sweeps, ctypes.byref(sw)))
        return t, sw.value

    def degree_levels(self):
        """Degree levels, Def. 5.  Returns (number of levels, level of each R)."""
        lv = np.zeros(self.num_r, dtype=np.int32)
        k = int(self._lib.orc_degree_levels(self._h, _ptr(lv)))
        if k < 0:
            _check(k)
        return k, lv


def _load_mt():
    global _mt
    with _lock:
        if _mt is not None:
            return _mt
        build()
        lib = ctypes.CDLL(_MT_PATH)
        i64, i32, vp, ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int
        lib.omt_create.argtypes = [i64, vp, vp, ci, ci, ctypes.POINTER(vp)]
        lib.omt_free.argtypes = [vp]
        lib.omt_free.restype = None
        lib.omt_num_r.argtypes = [vp]
        lib.omt_num_r.restype = i64
        lib.omt_num_incidences.argtypes = [vp]
        lib.omt_num_incidences.restype = i64
        lib.omt_snd.argtypes = [vp, vp, ci, i32, ci, vp, vp, vp]
        lib.omt_max_threads.restype = ci
        _mt = lib
        return lib


class ParallelSND:
    """SND (Alg. 2) on all host cores, for timing the CPU baseline: the
    oracle's arithmetic (Def. 4, H by sorting) with the loop over r-clique
    split over OpenMP threads, and its own incidence construction (Def. 1),
    also threaded.  (1,2) and (2,3).  The graph is validated by the
    single-threaded oracle first."""

    def __init__(self, row_ptr, col, r: int, threads: int = 0, validate: bool = True):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        if validate:
            Graph(self.row_ptr, self.col, r, r + 1, incidence=False)  # raises on a malformed graph
        lib = _load_mt()
        self._lib = lib
        self.threads = int(threads) if threads > 0 else int(lib.omt_max_threads())
        h = ctypes.c_void_p()
        _check(lib.omt_create(self.row_ptr.size - 1, _ptr(self.row_ptr), _ptr(self.col), r, self.threads,
                              ctypes.byref(h)))
        self._h = h
        self.r = r
        self.num_r = int(lib.omt_num_r(h))
        self.num_incidences = int(lib.omt_num_incidences(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.omt_free(h)
            self._h = None

    def snd(self, tau=None, max_sweeps: int = 1 << 30):
        """At most max_sweeps SND passes from d_s (or from tau).
        Returns (tau, sweeps, updating_sweeps, evaluations), as Graph.snd."""
        t = np.zeros(self.num_r, dtype=np.int32) if tau is None else \
            np.ascontiguousarray(np.asarray(tau, dtype=np.int32).copy())
        sw, up, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.omt_snd(self._h, _ptr(t), int(tau is None), int(max_sweeps), self.threads,
                                 ctypes.byref(sw), ctypes.byref(up), ctypes.byref(ev)))
        return t, sw.value, up.value, ev.value


def kendall_tau_b(x, y):
    """Kendall's tau-b of two integer sequences by visiting every pair
    (Section 5.2, Fig. 7).  Returns (tau_b, S, ties_x, ties_y); tau_b is NaN
    when either sequence is constant.  O(n^2)."""
    a = np.ascontiguousarray(x, dtype=np.int32)
    b = np.ascontiguousarray(y, dtype=np.int32)
    if a.shape != b.shape:
        raise ValueError("sequences differ in length")
    S, tx, ty = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    t = _load().orc_kendall_tau_b(_ptr(a), _ptr(b), a.size, ctypes.byref(S), ctypes.byref(tx), ctypes.byref(ty))
    return float(t), S.value, tx.value, ty.value


def decompose(row_ptr, col, r: int, s: int) -> np.ndarray:
    """kappa_s for every r-clique, canonical order (peeling, Alg. 1)."""
    return Graph(row_ptr, col, r, s, incidence=False).peel()


# ---------------------------------------------------------------------------
# Brute force, Lemma 1: kappa_s(R) is the largest minimum S-degree over the
# sub-complexes that contain R.  A sub-complex keeps a set X of r-cliques and
# every s-clique whose r-cliques all lie in X (Def. 5's closure rule).
# Pure Python; only for graphs with at most ~16 r-cliques.
# ---------------------------------------------------------------------------

def _adj_sets(row_ptr, col):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col[row_ptr[u]:row_ptr[u + 1]]) for u in range(n)]


def enumerate_cliques(row_ptr, col, k: int):
    """All k-cliques as sorted tuples, by brute force over vertex subsets of
    neighbourhoods (independent of the C enumeration)."""
    adj = _adj_sets(row_ptr, col)
    n = len(adj)
    out = []
    for combo in itertools.combinations(range(n), k):
        if all(b in adj[a] for a, b in itertools.combinations(combo, 2)):
            out.append(combo)
    return out


def brute_force_kappa(row_ptr, col, r: int, s: int, max_r: int = 16):
    """kappa_s by Lemma 1 over every subset of r-cliques (exponential)."""
    R = enumerate_cliques(row_ptr, col, r)
    S = enumerate_cliques(row_ptr, col, s)
    if len(R) > max_r:
        raise ValueError("too many r-cliques for brute force")
    rid = {t: i for i, t in enumerate(R)}
    members = [[rid[sub] for sub in itertools.combinations(t, r)] for t in S]
    best = [0] * len(R)
    for mask in range(1, 1 << len(R)):
        inside = [(mask >> i) & 1 for i in range(len(R))]
        deg = [0] * len(R)
        for mem in members:
            if all(inside[i] for i in mem):
                for i in mem:
                    deg[i] += 1
        delta = min(deg[i] for i in range(len(R)) if inside[i])
        for i in range(len(R)):
            if inside[i] and delta > best[i]:
                best[i] = delta
    return R, best


def naive_kappa(row_ptr, col, r: int, s: int):
    """kappa_s by repeated deletion: for each k, delete every r-clique with
    fewer than k s-cliques left until stable; kappa(R) = largest k at which R
    survives.  Pure Python, O(k * |R|^2)."""
    R = enumerate_cliques(row_ptr, col, r)
    S = enumerate_cliques(row_ptr, col, s)
    rid = {t: i for i, t in enumerate(R)}
    members = [[rid[sub] for sub in itertools.combinations(t, r)] for t in S]
    kappa = [0] * len(R)
    k = 1
    while True:
        alive = [True] * len(R)
        changed = True
        while changed:
            changed = False
            deg = [0] * len(R)
            for mem in members:
                if all(alive[i] for i in mem):
                    for i in mem:
                        deg[i] += 1
            for i in range(len(R)):
                if alive[i] and deg[i] < k:
                    alive[i] = False
                    changed = True
        if not any(alive):
            break
        for i in range(len(R)):
            if alive[i]:
                kappa[i] = k
        k += 1
    return R, kappa

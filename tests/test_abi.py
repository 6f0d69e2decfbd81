"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function include/nd.h declares; host-only calls work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1704_00386_gb300 import nd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(nd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = nd.load()
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(nd.SYMBOLS) == set(declared)


def test_host_only_calls():
    assert nd.abi_version() == 1
    assert nd.strerror(nd.ND_OK) == "ok"
    assert "unsupported" in nd.strerror(nd.ND_E_UNSUPPORTED_RS)
    lib = nd.load()
    assert isinstance(lib.nd_last_error(), bytes)


def test_host_buffers_need_the_gpu_too():
    """Host-buffer calls copy through the device; with no GPU they report an
    error instead of computing on the CPU (there is no CPU path)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    k = np.array([0, 1, 5], np.int32)
    with pytest.raises(nd.NDError):
        nd.truss_classic(k)
    with pytest.raises(nd.NDError):
        nd.kendall_tau_b(k, k)


def test_on_the_fly_flags_checked_before_touching_the_gpu():
    import ctypes
    import numpy as np
    lib = nd.load()
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    csr = nd._CSR(2, 2, nd._ptr(rp).value, nd._ptr(col).value, 0)
    h = ctypes.c_void_p()
    assert lib.nd_build_incidence_ex(ctypes.byref(csr), 2, 3, 6, None, ctypes.byref(h)) == nd.ND_E_INVAL
    assert lib.nd_build_incidence_ex(ctypes.byref(csr), 3, 4, nd.ND_BUILD_ON_THE_FLY, None,
                                     ctypes.byref(h)) == nd.ND_E_UNSUPPORTED_RS
    assert not h.value


def test_size_limits_checked_before_any_copy():
    """A k-truss input with 2^32 or more CSR entries (any r >= 2 with 2^32 or
    more edges) is refused from its header alone (the arrays are never read; a device pointer that is never
    dereferenced stands in for 16 GB of column indices)."""
    import ctypes
    import numpy as np
    lib = nd.load()
    rp = np.array([0, 0], np.int64)
    big = nd._CSR(1, 1 << 32, nd._ptr(rp).value, 0x1000, 1)
    h = ctypes.c_void_p()
    assert lib.nd_build_incidence(ctypes.byref(big), 2, 3, None, ctypes.byref(h)) == nd.ND_E_TOO_LARGE
    assert "2^32" in nd.load().nd_last_error().decode()
    bigger = nd._CSR(1, 1 << 33, nd._ptr(rp).value, 0x1000, 1)  # 2^32 edges: past the edge-id range
    assert lib.nd_build_incidence(ctypes.byref(bigger), 3, 4, None, ctypes.byref(h)) == nd.ND_E_TOO_LARGE
    assert not h.value


def test_rejects_bad_arguments_before_touching_the_gpu():
    import numpy as np
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, 1, 3)
    assert e.value.status == nd.ND_E_UNSUPPORTED_RS
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, 2, 2)
    assert e.value.status == nd.ND_E_INVAL
    lib = nd.load()
    out = ctypes.c_void_p()
    assert lib.nd_build_incidence(None, 1, 2, None, ctypes.byref(out)) == nd.ND_E_INVAL


def test_binding_has_no_cpu_fallback():
    src = open(os.path.join(ROOT, "paper_1704_00386_gb300", "nd.py")).read()
    assert "oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_1704_00386_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_1704_00386_gb300", f)).read()


def test_every_call_checks_its_arguments_before_touching_the_gpu():
    """Each entry point rejects a NULL handle, a negative size or a bad
    option with a status, before any CUDA call (none is made here: this runs
    with no GPU)."""
    lib = nd.load()
    INVAL = nd.ND_E_INVAL
    i32, i64, dbl, cint = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
    r = ctypes.byref
    assert lib.nd_incidence_info(None, r(i64), r(i64), r(cint)) == INVAL
    assert lib.nd_incidence_bytes(None, r(i64)) == INVAL
    assert lib.nd_r_cliques(None, None, 0, None) == INVAL
    assert lib.nd_s_degree(None, None, 0, None) == INVAL
    assert lib.nd_snd(None, None, 0, 10, r(i32), None) == INVAL
    assert lib.nd_and(None, None, 0, 1, 10, r(i32), r(i64), None) == INVAL
    assert lib.nd_iterate_k(None, 0, -1, None, 0, 0, r(i32), None) == INVAL   # negative k
    assert lib.nd_iterate_k(None, 0, 1, None, 0, 0, r(i32), None) == INVAL    # no handle
    assert lib.nd_and_partial(None, None, 0, 0, None, 10, r(i32), r(i64), None) == INVAL
    assert lib.nd_and_until(None, 0.5, None, 0, 10, r(i32), r(i64), r(cint), None) == INVAL
    assert lib.nd_autotune(None, 1, None, None, None) == INVAL
    assert lib.nd_last_passes(None, None, None, None, 0, r(i32)) == INVAL
    assert lib.nd_count_equal(None, None, -1, 0, r(i64), None) == INVAL
    assert lib.nd_count_equal(None, None, 0, 0, None, None) == INVAL            # no result slot
    assert lib.nd_truss_classic(None, -1, None, 0, None) == INVAL
    assert lib.nd_kendall_tau_b(None, None, -1, 0, r(dbl), None, None) == INVAL
    # batches: a negative count, or graphs missing
    h = ctypes.c_void_p()
    assert lib.nd_build_incidence_batch(None, -1, 1, 2, None, r(h), None) == INVAL
    assert lib.nd_build_incidence_batch(None, 2, 1, 2, None, r(h), None) == INVAL
    assert lib.nd_build_incidence_batch(None, 0, 2, 5, None, r(h), None) == nd.ND_E_UNSUPPORTED_RS
    # no build flag outside the documented ones, the high bit included
    import numpy as np
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    csr = nd._CSR(2, 2, nd._ptr(rp).value, nd._ptr(col).value, 0)
    assert lib.nd_build_incidence_ex(r(csr), 2, 3, 1 << 31, None, r(h)) == INVAL
    assert not h.value
    # the allocation-free core call: sizes first
    assert lib.nd_core_snd_noalloc(None, None, -1, 0, None, 10, r(i32), None) == INVAL
    assert lib.nd_core_snd_noalloc(None, None, (1 << 20) + 1, 0, None, 10, r(i32), None) == nd.ND_E_TOO_LARGE
    # n = 0 is the entry point's set-up call: it needs a device (none here)
    assert lib.nd_core_snd_noalloc(None, None, 0, 0, None, 10, r(i32), None) == nd.ND_E_CUDA
    # normalisation: sizes and pointers first
    nnz = ctypes.c_int64()
    assert lib.nd_normalize(None, None, -1, 5, 0, None, None, 0, r(nnz), None) == INVAL
    assert lib.nd_normalize(None, None, 3, 5, 0, None, None, 6, r(nnz), None) == INVAL     # no pairs given
    assert lib.nd_normalize(None, None, 0, 1 << 31, 0, None, None, 0, r(nnz), None) == nd.ND_E_TOO_LARGE
    assert lib.nd_normalize(None, None, 2, 0, 0, None, None, 4, r(nnz), None) == INVAL     # edges, no vertices
    # process-wide limits: values checked, defaults restored
    assert lib.nd_set_wait_limit(0.0) == INVAL
    assert lib.nd_set_wait_limit(-1.0) == INVAL
    assert lib.nd_set_wait_limit(600.0) == nd.ND_OK
    assert lib.nd_set_handle_memory_limit(-1) == INVAL
    assert lib.nd_set_handle_memory_limit(0) == nd.ND_OK
    # every status has a message; an unknown one says so
    for st in range(nd.ND_E_BUSY + 1):
        assert nd.strerror(st) != "unknown status"
    assert "handle" in nd.strerror(nd.ND_E_BUSY)
    assert lib.nd_strerror(999) == b"unknown status"

"""nd_core_snd_noalloc, the entry point that allocates nothing.

It is for callers that cannot allocate device memory when they call in:
their process has given the GPU's memory to another allocator up front, or
they cannot take the device synchronisation that cudaMalloc / cudaFree
imply.  Its only scratch is a fixed file-scope device array, shared by every
call, so these tests check that consecutive calls on different graphs give
exactly the core numbers of the allocating path (nd_build_incidence(g, 1, 2)
+ nd_snd) and of the CPU oracle -- integers, so the comparisons are exact --
that oversized graphs are refused, and that after the size-0 set-up call
two more calls change the device's free memory by nothing.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_VERTICES = 1 << 20


def _graphs():
    w = G.workload("chunglu_n2000_g2.5_d10")
    n, s, d = G.rmat(14, 16, seed=41)
    rp2, col2 = G.to_csr(n, s, d)
    rp3, col3 = G.hub_graph(3000, 6, seed=107)
    # largest first, then smaller ones: stale scratch from a previous call would show
    return [(rp2, col2), (w["row_ptr"], w["col"]), (rp3, col3), (rp2, col2)]


def _call_noalloc(lib, rp_d, col_d, out, max_iters=1 << 30):
    it = ctypes.c_int32(-1)
    st = lib.nd_core_snd_noalloc(ctypes.c_void_p(rp_d.data_ptr()), ctypes.c_void_p(col_d.data_ptr()),
                                 rp_d.numel() - 1, col_d.numel(), ctypes.c_void_p(out.data_ptr()),
                                 max_iters, ctypes.byref(it),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, it.value


def test_noalloc_matches_allocating_snd_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    lib = nd.load()
    for rp, col in _graphs():
        rp_d = torch.from_numpy(rp).cuda()
        col_d = torch.from_numpy(col).cuda()
        inc = nd.build_incidence(rp_d, col_d, 1, 2)
        want, want_iters = inc.snd()
        inc.free()
        out = torch.full((rp.size - 1,), -7, dtype=torch.int32, device="cuda")
        st, iters = _call_noalloc(lib, rp_d, col_d, out)
        assert st == nd.ND_OK, lib.nd_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(out, want)
        assert iters == want_iters


def test_noalloc_matches_the_oracle_directly():
    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    lib = nd.load()
    for rp, col in _graphs()[:3]:
        rp_d = torch.from_numpy(rp).cuda()
        col_d = torch.from_numpy(col).cuda()
        out = torch.full((rp.size - 1,), -7, dtype=torch.int32, device="cuda")
        st, _ = _call_noalloc(lib, rp_d, col_d, out)
        assert st == nd.ND_OK, lib.nd_last_error().decode()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.decompose(rp, col, 1, 2))


def test_noalloc_allocates_nothing_after_its_set_up_call():
    """A call with n = 0 loads the entry point's code and scratch array onto
    the device; after it, calls take no device memory: the free memory the
    driver reports is the same before and after two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    lib = nd.load()
    w = G.workload("chunglu_n2000_g2.5_d10")
    n, s, d = G.rmat(14, 16, seed=43)
    rp2, col2 = G.to_csr(n, s, d)
    args = []
    for rp, col in ((w["row_ptr"], w["col"]), (rp2, col2)):
        rp_d = torch.from_numpy(rp).cuda()
        col_d = torch.from_numpy(col).cuda()
        out = torch.empty(rp.size - 1, dtype=torch.int32, device="cuda")
        args.append((rp_d, col_d, out))
    it = ctypes.c_int32()
    assert lib.nd_core_snd_noalloc(None, None, 0, 0, None, 0, ctypes.byref(it), None) == nd.ND_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for rp_d, col_d, out in args:
        st, _ = _call_noalloc(lib, rp_d, col_d, out)
        assert st == nd.ND_OK, lib.nd_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_iteration_cap_and_size_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    lib = nd.load()
    rp, col = G.workload("chunglu_n2000_g2.5_d10")["row_ptr"], G.workload("chunglu_n2000_g2.5_d10")["col"]
    rp_d = torch.from_numpy(rp).cuda()
    col_d = torch.from_numpy(col).cuda()
    out = torch.empty(rp.size - 1, dtype=torch.int32, device="cuda")
    st, iters = _call_noalloc(lib, rp_d, col_d, out, max_iters=1)
    assert st == nd.ND_E_NOT_CONVERGED and iters == 1
    big = torch.zeros(MAX_VERTICES + 2, dtype=torch.int64, device="cuda")  # n = MAX + 1, no edges
    st, _ = _call_noalloc(lib, big, col_d, out)
    assert st == nd.ND_E_TOO_LARGE
    assert b"1048576" in lib.nd_last_error()
    ok = torch.zeros(MAX_VERTICES + 1, dtype=torch.int64, device="cuda")  # n = MAX exactly
    out2 = torch.full((MAX_VERTICES,), 5, dtype=torch.int32, device="cuda")
    st, _ = _call_noalloc(lib, ok, col_d[:0], out2)
    assert st == nd.ND_OK
    assert int(out2.abs().sum()) == 0  # isolated vertices: core number 0

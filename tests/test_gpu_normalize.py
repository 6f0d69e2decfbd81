"""nd_normalize: arbitrary vertex pairs -> the simple undirected CSR of
Section 2 (no self-loop, no repeated edge, symmetric, rows sorted).

The expected CSR comes from graphs.to_csr (numpy: drop loops, order each
pair, np.unique, symmetrise, sort), which holds none of the method's
arithmetic; the kernel path (a radix sort on the GPU) must give the same
bytes.  At full size the raw R-MAT scale-20 samples of the k-truss
workload go through nd_normalize and then the decomposition, whose kappa
must hash to the oracle's stored digest.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    return nd


def _pairs(n, m, seed, loops=0.05, repeats=0.3):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m, dtype=np.int64)
    dst = rng.integers(0, n, size=m, dtype=np.int64)
    k = int(loops * m)
    dst[:k] = src[:k]                                   # self-loops
    r = int(repeats * m)
    if r and m > r:
        pick = rng.integers(0, m - r, size=r)
        flip = rng.random(r) < 0.5                      # repeats in both directions
        src[m - r:] = np.where(flip, dst[pick], src[pick])
        dst[m - r:] = np.where(flip, src[pick], dst[pick])
    return src, dst


CASES = [
    (1, 0), (1, 5), (2, 1), (7, 40), (100, 700), (3000, 50_000), (70_000, 300_000),
    (1 << 16, 200_000),       # n a power of two: ids use every bit of their field
    ((1 << 16) + 1, 200_000),
    (5000, 4097),             # ragged sort tiles (4096 keys each)
]


@pytest.mark.parametrize("n,m", CASES)
@pytest.mark.parametrize("where", ["host", "device"])
def test_normalize_equals_the_plain_construction(n, m, where):
    nd = _nd()
    src, dst = _pairs(n, m, seed=n * 7 + m)
    want_rp, want_col = G.to_csr(n, src, dst)
    if where == "device":
        rp, col = nd.normalize(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
        rp, col = rp.cpu().numpy(), col.cpu().numpy()
    else:
        rp, col = nd.normalize(src, dst, n)
    assert rp.dtype == np.int64 and col.dtype == np.int32
    np.testing.assert_array_equal(rp, want_rp)
    np.testing.assert_array_equal(col, want_col)


def test_normalize_hub_rows_and_isolated_vertices():
    """A vertex adjacent to every other one (a row of 20,000 entries, spread
    over many sort tiles) next to isolated vertices and repeated stars."""
    nd = _nd()
    n = 40_000
    hub = np.zeros(20_000, np.int64)
    leaves = np.arange(1, 20_001, dtype=np.int64)
    src = np.concatenate([hub, leaves, leaves[::3]])
    dst = np.concatenate([leaves, hub, hub[: leaves[::3].size]])
    want = G.to_csr(n, src, dst)
    got = nd.normalize(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    np.testing.assert_array_equal(got[0].cpu().numpy(), want[0])
    np.testing.assert_array_equal(got[1].cpu().numpy(), want[1])
    assert int(got[0][-1]) == 40_000 and int(got[0][20_002] - got[0][20_001]) == 0


def test_normalize_rejects_bad_ids_and_short_output():
    import ctypes
    nd = _nd()
    lib = nd.load()
    src = np.array([0, 1, 2], np.int64)
    for bad in (np.array([1, 2, 3], np.int64), np.array([1, -1, 0], np.int64)):
        rp = np.zeros(4, np.int64)
        col = np.zeros(6, np.int32)
        nnz = ctypes.c_int64()
        st = lib.nd_normalize(nd._ptr(src), nd._ptr(bad), 3, 3, 0, nd._ptr(rp), nd._ptr(col), 6,
                              ctypes.byref(nnz), None)
        assert st == nd.ND_E_INVAL
        assert b"outside" in lib.nd_last_error()
    # a triangle needs 6 entries: capacity 5 is refused and the size reported
    dst = np.array([1, 2, 0], np.int64)
    rp = np.zeros(4, np.int64)
    col = np.zeros(5, np.int32)
    nnz = ctypes.c_int64()
    st = lib.nd_normalize(nd._ptr(src), nd._ptr(dst), 3, 3, 0, nd._ptr(rp), nd._ptr(col), 5, ctypes.byref(nnz),
                          None)
    assert st == nd.ND_E_INVAL and nnz.value == 6


def test_normalize_then_decompose_matches_the_oracle():
    """From raw pairs to kappa on the GPU: the normalised graph is a valid
    input, and its k-core, k-truss and (3,4) numbers equal the oracle's."""
    import oracle
    nd = _nd()
    n = 600
    s1, d1 = G.chung_lu(n, 2.3, 9.0, seed=31)
    s2, d2 = G.plant_cliques(n, 3, 8, 14, seed=32)
    src = np.concatenate([s1, s2, d1[:500]])            # repeats, reversed
    dst = np.concatenate([d1, d2, s1[:500]])
    rp, col = nd.normalize(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    rp_h, col_h = rp.cpu().numpy(), col.cpu().numpy()
    for r, s in ((1, 2), (2, 3), (3, 4)):
        inc = nd.build_incidence(rp, col, r, s)
        got, _ = inc.snd()
        inc.free()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.decompose(rp_h, col_h, r, s))


@pytest.mark.timeout(900)
def test_normalize_full_size_truss_workload():
    """The R-MAT scale-20 k-truss workload from its raw samples (16.8M pairs
    with loops and repeats): the CSR equals the plain construction, and the
    k-truss numbers of that CSR hash to the oracle's digest."""
    nd = _nd()
    with open(os.path.join(ROOT, "tests", "golden", "digests.json")) as f:
        gold = json.load(f)["rmat_s20_ef16"]
    n, src, dst = G.rmat(20, 16, seed=2)
    rp, col = nd.normalize(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    csr = hashlib.sha256(rp.cpu().numpy().astype("<i8").tobytes() + col.cpu().numpy().astype("<i4").tobytes())
    assert csr.hexdigest() == gold["csr_sha256"]   # the oracle digests' input graph, byte for byte
    want_rp, want_col = G.to_csr(n, src, dst)
    np.testing.assert_array_equal(rp.cpu().numpy(), want_rp)
    np.testing.assert_array_equal(col.cpu().numpy(), want_col)
    del want_rp, want_col
    assert int(rp[-1]) == gold["nnz"]
    inc = nd.build_incidence(rp, col, 2, 3)
    kappa, _ = inc.snd()
    inc.free()
    k = kappa.cpu().numpy()
    assert hashlib.sha256(np.ascontiguousarray(k, dtype="<i4").tobytes()).hexdigest() == gold["kappa_sha256"]

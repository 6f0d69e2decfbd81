"""k-core of R-MAT scale 26, edge factor 16 (about 1.07G samples, 1.8G CSR
entries): every core number from SND and AND on the GPU against the CPU
oracle's Batagelj-Zaversnik peeling of the same CSR.  The graph comes from the
counter-based torch generator (identical on CPU and GPU), built on the GPU
and copied to the host for the oracle."""
import numpy as np
import pytest

import oracle
from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_rmat_scale26_kcore_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    w = G.workload("rmat_core_s26_ef16")
    rp, col = w["row_ptr"], w["col"]
    assert rp.is_cuda and rp.numel() == (1 << 26) + 1
    inc = nd.build_incidence(rp, col, 1, 2)
    tau, iters = inc.snd()
    t_and, it_and, _ = inc.and_(notify=True)
    assert torch.equal(tau, t_and) and it_and <= iters
    got = tau.cpu().numpy()
    inc.free()
    rp_h = rp.cpu().numpy()
    col_h = col.cpu().numpy()
    del rp, col, w
    torch.cuda.empty_cache()
    want = oracle.decompose(rp_h, col_h, 1, 2)
    np.testing.assert_array_equal(got, want)


def test_large_kcore_symmetry_check_rejects_a_missing_reverse():
    """Large k-core inputs (2^26 CSR entries or more) check their symmetry by
    sorting the transposed pairs instead of searching each entry: one entry
    moved to an id its row lacks (the row stays sorted, every id stays in
    range) leaves two pairs without their reverse, and the build refuses it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    n, s, d = G.rmat_torch(22, 16, seed=9, device="cuda")
    rp, col = G.to_csr_torch(n, s, d)
    del s, d
    assert col.numel() >= (1 << 26)
    inc = nd.build_incidence(rp, col, 1, 2)       # the valid graph passes the check
    inc.free()
    rp_h = rp.cpu().numpy()
    col_h = col.cpu().numpy()
    # the first entry p of a row u whose next neighbour is at least 2 ids further on,
    # with col[p] + 1 != u: move it to col[p] + 1, which row u does not hold
    gap = (col_h[1:] - col_h[:-1]) >= 2
    row_of = np.repeat(np.arange(n), np.diff(rp_h))
    same_row = row_of[1:] == row_of[:-1]
    cand = np.nonzero(gap & same_row & (col_h[:-1] + 1 != row_of[:-1]))[0]
    p = int(cand[len(cand) // 2])
    bad = col.clone()
    bad[p] += 1
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, bad, 1, 2)
    assert e.value.status == nd.ND_E_INVAL
    assert "symmetric" in str(e.value)

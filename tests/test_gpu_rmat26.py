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

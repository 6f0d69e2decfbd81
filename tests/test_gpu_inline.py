"""The inline SND mode of the k-truss: once few edges change, each
incidence entry keeps 16-bit copies of its two edges' tau and the changed
edges push their new values between passes.  It must not change a single
value: the SND iterate after every pass (Alg. 2 is deterministic) equals
the oracle's, across the switch, and so do kappa and the pass count."""
import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    return nd


@pytest.mark.parametrize("scale,ef,seed", [(13, 16, 3), (15, 8, 4), (17, 4, 19)])
def test_inline_snd_follows_the_oracle_pass_by_pass(scale, ef, seed):
    import oracle
    nd = _nd()
    n, s, d = G.rmat(scale, ef, seed=seed)
    rp, col = G.to_csr(n, s, d)
    g = oracle.Graph(rp, col, 2, 3, incidence=True)
    kappa, sweeps, updating, _ = g.snd()
    inc = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), 2, 3)
    nd.prof_enable(True)
    got, iters = inc.snd()
    prof = nd.prof_read()
    nd.prof_enable(False)
    np.testing.assert_array_equal(got.cpu().numpy(), kappa)
    assert iters == updating
    assert "init_inline" in prof, "the run never switched to the inline mode"
    # every iterate, before and after the switch (which comes after a batch of 8 passes)
    tau = g.snd(max_sweeps=0)[0]
    for k in range(1, updating + 1):
        want = g.snd(tau=tau, max_sweeps=1)[0]
        step, _ = inc.iterate_k("snd", k)
        np.testing.assert_array_equal(step.cpu().numpy(), want, err_msg=f"pass {k}")
        tau = want
    # the handle goes on to AND with notification from d_s
    np.testing.assert_array_equal(inc.and_(notify=True)[0].cpu().numpy(), kappa)
    np.testing.assert_array_equal(inc.snd()[0].cpu().numpy(), kappa)   # and SND again, inline copies reused
    inc.free()

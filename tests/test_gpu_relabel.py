"""A k-truss build that renumbers the graph by degree class (graphs of
65,536 vertices or more): the handle works on internal vertex and edge ids,
and every call must still take and give the caller's ids.  Checked against
the oracle, which never relabels: the r-clique tuples, d_s, kappa by SND,
AND and AND-nn, the SND iterates tau_1 and tau_2 (deterministic, Alg. 2),
a restart from the oracle's tau_2 (Lemma 2), PartialAnd on a set of the
caller's edge ids, and the same through host buffers."""
import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    n, s, d = G.rmat(17, 4, seed=19)          # 131,072 vertices: above the relabelling threshold
    rp, col = G.to_csr(n, s, d)
    g = oracle.Graph(rp, col, 2, 3, incidence=True)
    return dict(rp=rp, col=col, g=g, kappa=g.peel(), tuples=g.r_cliques(), ds=g.s_degree(),
                tau1=g.snd(max_sweeps=1)[0], tau2=g.snd(max_sweeps=2)[0], tau3=g.snd(max_sweeps=3)[0])


def test_relabelled_truss_in_the_callers_ids(case):
    from paper_1704_00386_gb300 import nd
    rp_d = torch.from_numpy(case["rp"]).cuda()
    col_d = torch.from_numpy(case["col"]).cuda()
    inc = nd.build_incidence(rp_d, col_d, 2, 3)
    assert inc.num_r == case["g"].num_r and inc.num_incidences == case["g"].num_incidences
    np.testing.assert_array_equal(inc.r_cliques().cpu().numpy(), case["tuples"])
    np.testing.assert_array_equal(inc.s_degree().cpu().numpy(), case["ds"])
    kappa = case["kappa"]
    np.testing.assert_array_equal(inc.snd()[0].cpu().numpy(), kappa)
    np.testing.assert_array_equal(inc.and_(notify=True)[0].cpu().numpy(), kappa)
    np.testing.assert_array_equal(inc.and_(notify=False)[0].cpu().numpy(), kappa)
    np.testing.assert_array_equal(inc.iterate_k("snd", 1)[0].cpu().numpy(), case["tau1"])
    np.testing.assert_array_equal(inc.iterate_k("snd", 2)[0].cpu().numpy(), case["tau2"])
    t2 = torch.from_numpy(case["tau2"]).cuda()
    np.testing.assert_array_equal(inc.iterate_k("snd", 1, tau=t2)[0].cpu().numpy(), case["tau3"])
    # PartialAnd on every third edge of the caller's numbering
    members = np.arange(0, inc.num_r, 3, dtype=np.uint32)
    mask = np.zeros(inc.num_r, bool)
    mask[members] = True
    want, _, _, _ = case["g"].partial_and(mask)
    got, _, _ = inc.and_partial(torch.from_numpy(members.astype(np.int32)).cuda())
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    inc.free()


def test_relabelled_truss_through_host_buffers(case):
    from paper_1704_00386_gb300 import nd
    inc = nd.build_incidence(case["rp"], case["col"], 2, 3)
    np.testing.assert_array_equal(inc.r_cliques(), case["tuples"])
    np.testing.assert_array_equal(inc.snd()[0], case["kappa"])
    np.testing.assert_array_equal(inc.iterate_k("snd", 1, tau=case["tau2"])[0], case["tau3"])
    inc.free()

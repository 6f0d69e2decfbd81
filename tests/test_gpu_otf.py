"""The no-storage mode (ND_BUILD_ON_THE_FLY): no r-clique -> s-clique
incidence is kept, and every pass finds the triangles of each edge again, as
the paper's own implementation does (Section 4.1, "Time complexity";
Section 5).  Every result must equal the oracle's and the stored mode's
bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd as _nd
    _nd.load()
    return _nd


def _cases():
    out = {"toy": G.toy_core_graph(), "k9": G.complete_graph(9)}
    s, d = G.chung_lu(700, 2.3, 10.0, seed=201)
    out["chunglu700"] = G.to_csr(700, s, d)
    n, s, d = G.rmat(10, 8, seed=202)
    out["rmat10"] = G.to_csr(n, s, d)
    s1, d1 = G.chung_lu(900, 2.1, 6.0, seed=203)
    s2, d2 = G.plant_cliques(900, 5, 8, 30, seed=204)
    out["planted900"] = G.to_csr(900, np.concatenate([s1, s2]), np.concatenate([d1, d2]))
    out["hubs3000"] = G.hub_graph(3000, 6, seed=205)
    return out


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_truss_on_the_fly_bit_exact(nd, name):
    rp, col = CASES[name]
    inc = nd.build_incidence(rp, col, 2, 3, on_the_fly=True)
    ref = nd.build_incidence(rp, col, 2, 3)
    g = oracle.Graph(rp, col, 2, 3)
    assert inc.num_r == g.num_r and inc.num_incidences == g.num_incidences
    if g.num_r == 0:
        return
    np.testing.assert_array_equal(inc.s_degree(), g.s_degree())
    kap = g.peel()
    tau, iters = inc.snd()
    np.testing.assert_array_equal(tau, kap)
    assert iters == g.snd()[2]
    for notify in (True, False):
        ta, it_a, _ = inc.and_(notify=notify)
        np.testing.assert_array_equal(ta, kap)
        assert it_a <= iters
    for k in (1, 2, 3):
        np.testing.assert_array_equal(inc.iterate_k("snd", k)[0], g.snd(max_sweeps=k)[0])
        ta, _ = inc.iterate_k("and", k)
        assert (kap <= ta).all() and (ta <= inc.iterate_k("snd", k)[0]).all()
    # the same evaluations and changes per SND pass as the stored mode
    ref.snd()
    inc.snd()
    np.testing.assert_array_equal(np.stack(inc.last_passes()), np.stack(ref.last_passes()))
    # PartialAnd: members only
    members = np.arange(0, g.num_r, 3, dtype=np.uint32)
    np.testing.assert_array_equal(inc.and_partial(members)[0], ref.and_partial(members)[0])


def test_on_the_fly_keeps_no_incidence(nd):
    rp, col = CASES["planted900"]
    inc = nd.build_incidence(rp, col, 2, 3, on_the_fly=True)
    ref = nd.build_incidence(rp, col, 2, 3)
    # the stored mode holds 8 B per incidence more (the on-the-fly handle keeps
    # a 16-byte placeholder in its place)
    assert ref.incidence_bytes() - inc.incidence_bytes() >= 8 * ref.num_incidences - 16


def test_on_the_fly_exact_path_for_huge_tau(nd):
    """Two adjacent hubs with 66,000 common neighbours: in the first pass the
    hub edge has tau = 66,000 > 65,535 and gathers exact int32 values."""
    fan = 66000
    w = np.arange(2, fan + 2)
    src = np.concatenate([[0], np.zeros(fan, np.int64), np.ones(fan, np.int64), w])
    dst = np.concatenate([[1], w, w, np.roll(w, -1)])
    rp, col = G.to_csr(fan + 2, src, dst)
    inc = nd.build_incidence(rp, col, 2, 3, on_the_fly=True)
    ref = nd.build_incidence(rp, col, 2, 3)
    for k in (1, 2):
        np.testing.assert_array_equal(inc.iterate_k("snd", k)[0], ref.iterate_k("snd", k)[0])
    np.testing.assert_array_equal(inc.snd()[0], ref.snd()[0])
    np.testing.assert_array_equal(inc.and_()[0], ref.snd()[0])


def test_on_the_fly_core_and_unsupported(nd):
    rp, col = CASES["chunglu700"]
    a = nd.build_incidence(rp, col, 1, 2, on_the_fly=True)
    b = nd.build_incidence(rp, col, 1, 2)
    np.testing.assert_array_equal(a.snd()[0], b.snd()[0])
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, 3, 4, on_the_fly=True)
    assert e.value.status == nd.ND_E_UNSUPPORTED_RS

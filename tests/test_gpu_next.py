"""The paper's query-driven and early-stopping tools on the GPU:

* PartialAnd (end of Section 4.3; ego networks, Section 5.4) against the CPU
  oracle's PartialAnd, bit for bit (the restricted iteration has one fixed
  point whatever the order);
* the active-ratio stopping rule (Section 5.2, Fig. 9): kappa <= tau <= d_s
  and no more work than the full run;
* the accuracy count used for the paper's accuracy curves.
"""
import numpy as np
import pytest

import oracle
from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RS = [(1, 2), (2, 3), (3, 4)]


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd as _nd
    _nd.load()
    return _nd


def _graphs():
    s1, d1 = G.chung_lu(800, 2.1, 6.0, seed=104)
    s2, d2 = G.plant_cliques(800, 6, 8, 22, seed=105)
    yield G.to_csr(800, np.concatenate([s1, s2]), np.concatenate([d1, d2]))
    yield G.hub_graph(1500, 4, seed=71)


@pytest.mark.parametrize("rs", RS)
def test_partial_and_matches_oracle(nd, rs):
    rng = np.random.default_rng(31)
    for rp, col in _graphs():
        inc = nd.build_incidence(rp, col, *rs)
        g = oracle.Graph(rp, col, *rs)
        if g.num_r == 0:
            continue
        for frac in (0.0, 0.05, 0.3, 1.0):
            mask = rng.random(g.num_r) < frac if frac < 1.0 else np.ones(g.num_r, bool)
            ids = np.flatnonzero(mask).astype(np.uint32)
            want = g.partial_and(mask)[0]
            got, _, _ = inc.and_partial(ids)
            np.testing.assert_array_equal(got, want)
        full, _, _ = inc.and_partial(np.arange(g.num_r, dtype=np.uint32))
        np.testing.assert_array_equal(full, g.peel())


def test_partial_and_ego_networks(nd):
    rp, col = next(_graphs())
    # (1,2): a vertex and its neighbours; (2,3): an edge and the edges sharing a triangle with it
    inc1 = nd.build_incidence(rp, col, 1, 2)
    g1 = oracle.Graph(rp, col, 1, 2)
    for u in (0, 5, 123):
        mask = np.zeros(g1.num_r, bool)
        mask[u] = True
        mask[col[rp[u]:rp[u + 1]]] = True
        got, _, _ = inc1.and_partial(np.flatnonzero(mask).astype(np.uint32))
        np.testing.assert_array_equal(got, g1.partial_and(mask)[0])
        assert got[u] >= g1.peel()[u]
    inc2 = nd.build_incidence(rp, col, 2, 3)
    g2 = oracle.Graph(rp, col, 2, 3)
    edges = {tuple(t): i for i, t in enumerate(g2.r_cliques().tolist())}
    adj = [set(col[rp[x]:rp[x + 1]].tolist()) for x in range(rp.size - 1)]
    for e in list(edges.values())[:40:7]:
        a, b = g2.r_cliques()[e]
        mask = np.zeros(g2.num_r, bool)
        mask[e] = True
        for w in adj[a] & adj[b]:
            mask[edges[(min(a, w), max(a, w))]] = True
            mask[edges[(min(b, w), max(b, w))]] = True
        got, _, _ = inc2.and_partial(np.flatnonzero(mask).astype(np.uint32))
        np.testing.assert_array_equal(got, g2.partial_and(mask)[0])


def test_partial_and_device_ids_and_bad_id(nd):
    rp, col = next(_graphs())
    dev = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), 2, 3)
    ids = torch.arange(0, dev.num_r, 3, dtype=torch.int32, device="cuda")
    got, _, _ = dev.and_partial(ids)
    mask = np.zeros(dev.num_r, bool)
    mask[::3] = True
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.Graph(rp, col, 2, 3).partial_and(mask)[0])
    with pytest.raises(nd.NDError) as e:
        dev.and_partial(torch.tensor([dev.num_r], dtype=torch.int32, device="cuda"))
    assert e.value.status == nd.ND_E_INVAL


@pytest.mark.parametrize("rs", RS)
def test_active_ratio_rule(nd, rs):
    n, s, d = G.rmat(13, 16, seed=77)
    rp, col = G.to_csr(n, s, d)
    inc = nd.build_incidence(rp, col, *rs)
    if inc.num_r == 0:
        return
    kap, it_full, ev_full = inc.and_(notify=True)
    ds = inc.s_degree()
    for ratio in (0.4, 0.1):
        tau, it, ev, stopped = inc.and_until(ratio)
        assert (kap <= tau).all() and (tau <= ds).all()
        assert ev <= ev_full
        if ratio == 0.4:
            # the late notified passes evaluate few r-cliques: the rule fires
            # (with every pass evaluating all of them, as without notification, it could not)
            assert stopped and it <= it_full
        if stopped:
            _, evals = inc.last_passes()
            assert evals[-1] < ratio * inc.num_r + (ds == 0).sum() + 1
        else:  # the run ended by converging: the result is kappa itself
            np.testing.assert_array_equal(tau, kap)
    tau0, _, _, stopped0 = inc.and_until(0.0)
    assert not stopped0
    np.testing.assert_array_equal(tau0, kap)


def test_count_equal(nd):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 5, size=100003).astype(np.int32)
    b = rng.integers(0, 5, size=100003).astype(np.int32)
    want = int((a == b).sum())
    assert nd.count_equal(a, b) == want
    assert nd.count_equal(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) == want
    assert nd.count_equal(a[:0], b[:0]) == 0

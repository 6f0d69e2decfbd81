"""Batched decomposition (nd_build_incidence_batch): many independent graphs
as one disjoint union, processed in one launch per pass.  Each graph's slice
must equal the CPU oracle's kappa and the single-graph CUDA result, bit for
bit, for every (r,s) and both host and device inputs."""
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


def _batch():
    gs = [(rp, col) for rp, col, _ in G.batch_graphs(24, seed=9, n_lo=30, n_hi=1500)]
    gs.insert(3, (np.zeros(1, np.int64), np.zeros(0, np.int32)))       # empty graph
    gs.insert(7, (np.zeros(5, np.int64), np.zeros(0, np.int32)))       # isolated vertices
    gs.append(G.complete_graph(9))
    return gs


BATCH = _batch()


@pytest.mark.parametrize("rs", [(1, 2), (2, 3), (3, 4)])
@pytest.mark.parametrize("where", ["host", "device"])
def test_batch_slices_match_oracle(nd, rs, where):
    gs = BATCH
    if where == "device":
        gs = [(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()) for rp, col in BATCH]
    inc, offs = nd.build_incidence_batch(gs, *rs)
    assert offs[0] == 0 and offs[-1] == inc.num_r
    tau, _ = inc.snd()
    ta, _, _ = inc.and_(notify=True)
    tau = tau.cpu().numpy() if where == "device" else tau
    ta = ta.cpu().numpy() if where == "device" else ta
    np.testing.assert_array_equal(tau, ta)
    for i, (rp, col) in enumerate(BATCH):
        want = oracle.decompose(rp, col, *rs)
        got = tau[offs[i]:offs[i + 1]]
        np.testing.assert_array_equal(got, want, err_msg=f"graph {i}")


def test_batch_equals_single_graph_runs(nd):
    inc, offs = nd.build_incidence_batch(BATCH, 2, 3)
    tuples = inc.r_cliques()
    tau, _ = inc.snd()
    base = 0
    for i, (rp, col) in enumerate(BATCH):
        single = nd.build_incidence(rp, col, 2, 3)
        assert single.num_r == offs[i + 1] - offs[i]
        if single.num_r:
            np.testing.assert_array_equal(single.snd()[0], tau[offs[i]:offs[i + 1]])
            np.testing.assert_array_equal(single.r_cliques() + base, tuples[offs[i]:offs[i + 1]])
        base += rp.size - 1


def test_batch_rejects_bad_part(nd):
    rp, col = G.toy_core_graph()
    bad = col.copy()
    bad[0] = 40                      # outside its own graph's vertex range
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence_batch([G.complete_graph(5), (rp, bad)], 1, 2)
    assert e.value.status == nd.ND_E_INVAL
    with pytest.raises(ValueError):
        nd.build_incidence_batch([(rp, col), (torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())], 1, 2)


@pytest.mark.parametrize("rs", [(1, 2), (2, 3)])
@pytest.mark.parametrize("mode", ["snd", "and_nn"])
def test_batch_stops_each_graph_where_its_own_run_stops(nd, rs, mode):
    """A graph whose pass changed nothing has converged (its tau is a fixed
    point), so a batch skips it from then on, as its own run would have
    stopped: the launched evaluations of the batch are exactly the sum of the
    single-graph runs' (d_s = 0 rows are never launched), and every slice
    equals its own run's result and the oracle's kappa."""
    inc, offs = nd.build_incidence_batch(BATCH, *rs)
    if mode == "snd":
        tau, iters = inc.snd()
    else:
        tau, iters, _ = inc.and_(notify=False)
    _, ev_b, inc_b = inc.last_passes(with_incidences=True)
    ds = inc.s_degree()
    launched_b = int(ev_b.sum()) - int((ds == 0).sum())   # the batch counts its d_s = 0 rows once
    launched, incidences, longest, longest_snd = 0, 0, 0, 0
    for i, (rp, col) in enumerate(BATCH):
        single = nd.build_incidence(rp, col, *rs)
        if single.num_r == 0:
            continue
        if mode == "snd":
            t, it = single.snd()
        else:
            t, it, _ = single.and_(notify=False)
        _, ev, ic = single.last_passes(with_incidences=True)
        zeros = int((single.s_degree() == 0).sum())
        launched += int(ev.sum()) - zeros * len(ev)
        incidences += int(ic.sum())
        longest = max(longest, it)
        longest_snd = max(longest_snd, single.snd()[1])
        np.testing.assert_array_equal(tau[offs[i]:offs[i + 1]], t, err_msg=f"graph {i}")
        np.testing.assert_array_equal(t, oracle.decompose(rp, col, *rs), err_msg=f"graph {i}")
        single.free()
    if mode == "snd":  # deterministic: the same rows in the same passes
        assert iters == longest
        assert launched_b == launched
        assert int(inc_b.sum()) == incidences
    else:
        # in place, the order inside a pass differs between the batch and the
        # single runs, and with it the number of passes; AND never needs more
        # passes than SND (Thm. 3 with in-place reads)
        assert iters <= longest_snd
    inc.free()

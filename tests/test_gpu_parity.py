"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integers throughout, so every comparison is bit-exact: r-clique tuples, d_s,
kappa_s from SND / AND / AND-nn, the SND iterates tau_k (deterministic,
Alg. 2) and iteration counts.  AND iterates are schedule-dependent and are
checked against the bounds kappa <= tau_AND_k <= tau_SND_k.
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


def _cases():
    out = {}
    out["toy"] = G.toy_core_graph()
    out["k7"] = G.complete_graph(7)
    s, d = G.chung_lu(600, 2.3, 9.0, seed=101)
    out["chunglu600"] = G.to_csr(600, s, d)
    i, j = G.erdos_renyi(500, 12 / 499, seed=102)
    out["er500"] = G.to_csr(500, i, j)
    n, s, d = G.rmat(10, 8, seed=103)
    out["rmat10"] = G.to_csr(n, s, d)
    # planted cliques over a sparse background: deep (3,4) nuclei, wide tails
    s1, d1 = G.chung_lu(800, 2.1, 6.0, seed=104)
    s2, d2 = G.plant_cliques(800, 6, 8, 22, seed=105)
    out["planted800"] = G.to_csr(800, np.concatenate([s1, s2]), np.concatenate([d1, d2]))
    # an edge in > 1024 triangles (CTA bucket for (2,3)) and a vertex of
    # degree > 1024 (CTA bucket for (1,2)), with a clique among the fan
    fan = 1300
    src = [0] * fan + [1] * fan + [0]
    dst = list(range(2, fan + 2)) + list(range(2, fan + 2)) + [1]
    a, b = np.triu_indices(40, 1)
    src += list(a + 2)
    dst += list(b + 2)
    out["book1300"] = G.to_csr(fan + 2, src, dst)
    out["hubs3000"] = G.hub_graph(3000, 6, seed=107)
    # closed forms: K_12 minus a perfect matching (kappa = d_s everywhere), a
    # wheel (core 3, truss 1, no 4-clique) and a windmill of 7 triangles
    half = 6
    cp = [(u, v) for u in range(2 * half) for v in range(u + 1, 2 * half) if v != u + half]
    out["cocktail12"] = G.to_csr(2 * half, [a for a, _ in cp], [b for _, b in cp])
    rim = 13
    wheel = [(0, i) for i in range(1, rim + 1)] + [(i, i % rim + 1) for i in range(1, rim + 1)]
    out["wheel13"] = G.to_csr(rim + 1, [a for a, _ in wheel], [b for _, b in wheel])
    wind = [p for i in range(7) for p in ((0, 1 + 2 * i), (0, 2 + 2 * i), (1 + 2 * i, 2 + 2 * i))]
    out["windmill7"] = G.to_csr(15, [a for a, _ in wind], [b for _, b in wind])
    return out


CASES = _cases()


def _run_all(nd, rp, col, r, s):
    inc = nd.build_incidence(rp, col, r, s)
    g = oracle.Graph(rp, col, r, s)
    return inc, g


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("rs", RS)
def test_small_graphs_bit_exact(nd, name, rs):
    rp, col = CASES[name]
    inc, g = _run_all(nd, rp, col, *rs)
    assert inc.num_r == g.num_r
    assert inc.q == g.q
    assert inc.num_incidences == g.num_incidences
    if g.num_r == 0:
        return
    np.testing.assert_array_equal(inc.r_cliques(), g.r_cliques())
    np.testing.assert_array_equal(inc.s_degree(), g.s_degree())
    kap = g.peel()
    tau, iters = inc.snd()
    np.testing.assert_array_equal(tau, kap)
    assert iters == g.snd()[2]  # SND is deterministic: same number of updating passes
    for notify in (True, False):
        t2, it2, ev2 = inc.and_(notify=notify)
        np.testing.assert_array_equal(t2, kap)
        assert it2 <= iters
        assert ev2 >= g.num_r
    for k in (1, 2, 3):
        tk, _ = inc.iterate_k("snd", k)
        np.testing.assert_array_equal(tk, g.snd(max_sweeps=k)[0])
        ta, _ = inc.iterate_k("and", k)
        assert (kap <= ta).all() and (ta <= tk).all()
        tn, _ = inc.iterate_k("and_nn", k)
        assert (kap <= tn).all() and (tn <= tk).all()


def test_toy_traces(nd):
    rp, col = G.toy_core_graph()
    inc = nd.build_incidence(rp, col, 1, 2)
    assert inc.iterate_k("snd", 1)[0].tolist() == [2, 2, 2, 2, 1, 1]
    assert inc.iterate_k("snd", 2)[0].tolist() == [1, 2, 2, 2, 1, 1]
    tau, iters = inc.snd()
    assert tau.tolist() == [1, 2, 2, 2, 1, 1] and iters == 2
    ch, ev = inc.last_passes()
    assert ch.tolist() == [2, 1, 0] and ev.tolist() == [6, 6, 6]


def test_device_tensors_and_host_arrays_agree(nd):
    rp, col = CASES["planted800"]
    for r, s in RS:
        host = nd.build_incidence(rp, col, r, s)
        dev = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), r, s)
        th, _ = host.snd()
        td, _ = dev.snd()
        assert isinstance(td, torch.Tensor) and td.is_cuda
        np.testing.assert_array_equal(th, td.cpu().numpy())
        ta, _, _ = dev.and_()
        np.testing.assert_array_equal(th, ta.cpu().numpy())
        np.testing.assert_array_equal(host.r_cliques(), dev.r_cliques().cpu().numpy())


def test_resume_from_saved_tau(nd):
    rp, col = CASES["rmat10"]
    inc = nd.build_incidence(rp, col, 2, 3)
    full, _ = inc.snd()
    mid, _ = inc.iterate_k("snd", 2)
    resumed, _ = inc.iterate_k("snd", 1 << 20, tau=mid)
    np.testing.assert_array_equal(resumed, full)
    resumed_and, _ = inc.iterate_k("and", 1 << 20, tau=mid)
    np.testing.assert_array_equal(resumed_and, full)


def test_iteration_cap_reports_not_converged(nd):
    rp, col = CASES["rmat10"]
    inc = nd.build_incidence(rp, col, 2, 3)
    _, iters = inc.snd()
    assert iters >= 2
    with pytest.raises(nd.NDError) as e:
        inc.snd(max_iters=1)
    assert e.value.status == nd.ND_E_NOT_CONVERGED


def test_empty_and_degenerate_graphs(nd):
    empty_rp, empty_col = np.zeros(1, np.int64), np.zeros(0, np.int32)
    for r, s in RS:
        inc = nd.build_incidence(empty_rp, empty_col, r, s)
        assert inc.num_r == 0
        assert inc.snd()[0].size == 0
    iso = np.zeros(9, np.int64)
    inc = nd.build_incidence(iso, empty_col, 1, 2)
    assert inc.snd()[0].tolist() == [0] * 8
    assert inc.and_()[0].tolist() == [0] * 8
    rp, col = G.cycle_graph(9)
    assert (nd.build_incidence(rp, col, 1, 2).snd()[0] == 2).all()
    assert (nd.build_incidence(rp, col, 2, 3).snd()[0] == 0).all()
    assert nd.build_incidence(rp, col, 3, 4).num_r == 0
    rp, col = G.star_graph(3000)  # hub of degree 3000: CTA bucket
    assert (nd.build_incidence(rp, col, 1, 2).and_()[0] == 1).all()


def test_closed_form_cliques(nd):
    for k in (4, 9, 33, 70):
        rp, col = G.complete_graph(k)
        for r, s in RS:
            inc = nd.build_incidence(rp, col, r, s)
            assert (inc.snd()[0] == k - r).all()
            assert (inc.and_()[0] == k - r).all()


@pytest.mark.parametrize("bad", ["unsorted", "asymmetric", "selfloop", "range", "rowptr"])
def test_malformed_graph_rejected(nd, bad):
    rp, col = G.toy_core_graph()
    rp = rp.copy()
    col = col.copy()
    if bad == "unsorted":
        col[2], col[3] = col[3], col[2]
    elif bad == "asymmetric":
        col[0] = 2                  # a lists c, but c does not list a
    elif bad == "selfloop":
        col[0] = 0
    elif bad == "range":
        col[0] = 99
    elif bad == "rowptr":
        rp[3] = 100
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, 1, 2)
    assert e.value.status == nd.ND_E_INVAL


def test_truss_with_high_out_degree_sources(nd):
    """Long oriented lists next to short ones.  A K_530 (every vertex 529
    neighbours: ids break the ties of the degree orientation, so the first
    vertices have out-degree above 512, and every edge lies in 528
    triangles) disjoint from a Chung-Lu graph of 3,000 vertices.  Closed
    form on the clique (truss number 528 for every edge), the oracle on the
    rest."""
    k = 530
    rest_rp, rest_col = G.to_csr(3000, *G.chung_lu(3000, 2.2, 10.0, seed=111))
    a, b = np.triu_indices(k, 1)
    src = np.concatenate([a, k + np.repeat(np.arange(3000), np.diff(rest_rp))])
    dst = np.concatenate([b, k + rest_col.astype(np.int64)])
    rp, col = G.to_csr(k + 3000, src, dst)
    want_rest = oracle.decompose(rest_rp, rest_col, 2, 3)
    m_clique = k * (k - 1) // 2
    for on_device in (False, True):
        args = (torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()) if on_device else (rp, col)
        inc = nd.build_incidence(*args, 2, 3)
        assert inc.num_r == m_clique + len(want_rest)
        ds = inc.s_degree()
        ds = ds.cpu().numpy() if on_device else ds
        assert (ds[:m_clique] == k - 2).all()
        for tau in (inc.snd()[0], inc.and_(notify=True)[0]):
            tau = tau.cpu().numpy() if on_device else tau
            assert (tau[:m_clique] == k - 2).all()      # edges (u, v), u < v < 530 come first
            np.testing.assert_array_equal(tau[m_clique:], want_rest)
        inc.free()


@pytest.mark.parametrize("rs", RS)
def test_overlapping_long_rows_rejected(nd, rs):
    """Long rows are listed before validation into arrays sized for disjoint
    rows; offsets whose rows overlap (every other row runs backwards, so
    each forward row spans the whole of col) must come back as ND_E_INVAL
    with nothing written past those arrays."""
    n, span = 7, 4100
    rp = np.array([0 if u % 2 == 0 else span for u in range(n)] + [span], np.int64)
    col = (np.arange(span) % n).astype(np.int32)
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, *rs)
    assert e.value.status == nd.ND_E_INVAL


def test_rows_past_the_16_bit_copy(nd):
    """A book of 70,000 pages: spine edge (0,1) in 70,000 triangles and two
    spine vertices of degree 70,001, so the first pass evaluates them with
    tau above 65,535, where the gathers read exact int32 values instead of
    the saturated 16-bit copy.  Closed forms (the oracle's linear merges with
    the spine rows would take minutes): every vertex in the 2-core, every
    edge in exactly the 1-truss (one triangle each off the spine), and no
    4-clique."""
    pages = 70000
    w = np.arange(2, pages + 2)
    rp, col = G.to_csr(pages + 2, np.concatenate([[0], np.zeros(pages, int), np.ones(pages, int)]),
                       np.concatenate([[1], w, w]))
    core = nd.build_incidence(rp, col, 1, 2)
    assert (core.s_degree()[:2] == pages + 1).all()
    assert (core.snd()[0] == 2).all() and (core.and_()[0] == 2).all()
    for on_the_fly in (False, True):
        truss = nd.build_incidence(rp, col, 2, 3, on_the_fly=on_the_fly)
        assert truss.num_r == 2 * pages + 1
        ds = truss.s_degree()
        assert ds[0] == pages and (ds[1:] == 1).all()      # edge (0,1) comes first
        tau, iters = truss.snd()
        assert (tau == 1).all() and iters == 1
        assert (truss.and_()[0] == 1).all()
    nucleus = nd.build_incidence(rp, col, 3, 4)
    assert nucleus.num_r == pages and (nucleus.snd()[0] == 0).all()


def _csr_of_lists(lists):
    rp = np.concatenate([[0], np.cumsum([len(l) for l in lists])]).astype(np.int64)
    col = np.concatenate([np.asarray(l, np.int32) for l in lists]).astype(np.int32)
    return rp, col


@pytest.mark.parametrize("bad", ["unsorted", "asymmetric_below", "asymmetric_above", "selfloop"])
def test_malformed_long_row_rejected(nd, bad):
    """Rows longer than 4,096 entries are validated in segments by a second
    launch; their faults must be found all the same.  A star: hub 0 and
    6,000 leaves, plus a path through the leaves so that (2,3) has work."""
    n = 6001
    lists = [list(range(1, n))] + [[0] for _ in range(1, n)]
    for leaf in range(1, n - 1):
        lists[leaf].append(leaf + 1)
        lists[leaf + 1].append(leaf)
    lists = [sorted(l) for l in lists]
    good_rp, good_col = _csr_of_lists(lists)
    assert nd.build_incidence(good_rp, good_col, 2, 3).num_r == len(good_col) // 2
    if bad == "unsorted":
        lists[0][100], lists[0][101] = lists[0][101], lists[0][100]
    elif bad == "asymmetric_above":
        lists[4000].remove(0)        # the hub lists leaf 4000, which no longer lists it
    elif bad == "asymmetric_below":
        lists[0].remove(4000)        # leaf 4000 lists the hub, which no longer lists it
    elif bad == "selfloop":
        lists[0] = [0] + lists[0]    # the hub lists itself
    rp, col = _csr_of_lists(lists)
    with pytest.raises(nd.NDError) as e:
        nd.build_incidence(rp, col, 2, 3)
    assert e.value.status == nd.ND_E_INVAL


def test_core_of_a_relabelled_graph(nd):
    """k-core handles of 65,536 vertices or more keep their vertices in
    degree-class order inside; every output, d_s, a caller's tau and
    PartialAnd member ids stay in the caller's ids."""
    n = 70000
    s1, d1 = G.chung_lu(n, 2.2, 8.0, seed=301)
    rp, col = G.to_csr(n, s1, d1)
    inc = nd.build_incidence(rp, col, 1, 2)
    g = oracle.Graph(rp, col, 1, 2)
    np.testing.assert_array_equal(inc.s_degree(), g.s_degree())
    np.testing.assert_array_equal(inc.r_cliques(), g.r_cliques())
    kap = g.peel()
    tau, iters = inc.snd()
    np.testing.assert_array_equal(tau, kap)
    assert iters == g.snd()[2]
    np.testing.assert_array_equal(inc.and_()[0], kap)
    t2 = g.snd(max_sweeps=2)[0]
    np.testing.assert_array_equal(inc.iterate_k("snd", 2)[0], t2)
    np.testing.assert_array_equal(inc.iterate_k("snd", 1 << 20, tau=t2)[0], kap)  # resume from caller ids
    members = np.arange(0, n, 7, dtype=np.uint32)
    mask = np.zeros(n, bool)
    mask[members] = True
    np.testing.assert_array_equal(inc.and_partial(members)[0], g.partial_and(mask)[0])
    dev = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), 1, 2)
    np.testing.assert_array_equal(dev.snd()[0].cpu().numpy(), kap)
    np.testing.assert_array_equal(dev.s_degree().cpu().numpy(), g.s_degree())


def test_classic_truss_device(nd):
    k = torch.tensor([0, 3, 7], dtype=torch.int32, device="cuda")
    assert nd.truss_classic(k).cpu().tolist() == [2, 5, 9]
    assert nd.truss_classic(np.array([0, 1, 5], np.int32)).tolist() == [2, 3, 7]


def test_kendall_tau_b_against_oracle(nd):
    """nd_kendall_tau_b (2D histogram, suffix sums) equals the oracle's pair
    loop exactly in its counts, on SND iterates against kappa (Section 5.2,
    Fig. 7), with and without ties and offsets."""
    rp, col = CASES["planted800"]
    for r, s in RS:
        inc = nd.build_incidence(rp, col, r, s)
        kap, _ = inc.snd()
        for k in (1, 2, 4):
            tk, _ = inc.iterate_k("snd", k)
            want = oracle.kendall_tau_b(tk, kap)
            got = nd.kendall_tau_b(tk, kap, with_counts=True)
            assert got[1:] == want[1:]
            assert got[0] == pytest.approx(want[0], abs=1e-12) or (np.isnan(got[0]) and np.isnan(want[0]))
            dev = nd.kendall_tau_b(torch.from_numpy(tk).cuda(), torch.from_numpy(kap).cuda())
            assert dev == got[0] or (np.isnan(dev) and np.isnan(got[0]))
    rng = np.random.default_rng(11)
    a = rng.integers(-40, 300, 5000).astype(np.int32)   # negative values: shifted histogram
    b = (a // 7 + rng.integers(0, 30, 5000)).astype(np.int32)
    want = oracle.kendall_tau_b(a, b)
    got = nd.kendall_tau_b(a, b, with_counts=True)
    assert got[1:] == want[1:]
    assert np.isnan(nd.kendall_tau_b(np.zeros(9, np.int32), a[:9]))  # constant: undefined
    assert np.isnan(nd.kendall_tau_b(a[:1], b[:1]))
    with pytest.raises(nd.NDError) as e:
        nd.kendall_tau_b(np.array([0, 1 << 20], np.int32), np.array([0, 1 << 20], np.int32))
    assert e.value.status == nd.ND_E_TOO_LARGE


def test_autotune_changes_speed_not_results(nd):
    rp, col = CASES["hubs3000"]
    for r, s in RS:
        inc = nd.build_incidence(rp, col, r, s)
        want, iters = inc.snd()
        thr, ms = inc.autotune(passes=2)
        assert thr[0] in (4, 8) and thr[1] in (32, 64) and thr[2] in (256, 1024, 2048, 8192)
        assert ms > 0
        got, iters2 = inc.snd()
        np.testing.assert_array_equal(got, want)
        assert iters2 == iters
        np.testing.assert_array_equal(inc.and_()[0], want)
        again = nd.build_incidence(rp, col, r, s)   # starts from the cached thresholds
        np.testing.assert_array_equal(again.snd()[0], want)


def test_long_rows_with_two_huge_endpoints(nd):
    """(2,3) rows are ordered by their third vertex with one bit per entry of
    the shorter adjacency list; an edge whose endpoints both have more than
    16,384 neighbours takes the global-scratch path.  Two adjacent hubs share
    66,000 neighbours, which form a cycle: the hub edge is in 66,000
    triangles, every other edge in 1-3."""
    fan = 66000
    w = np.arange(2, fan + 2)
    src = np.concatenate([[0], np.zeros(fan, np.int64), np.ones(fan, np.int64), w])
    dst = np.concatenate([[1], w, w, np.roll(w, -1)])
    rp, col = G.to_csr(fan + 2, src, dst)
    inc = nd.build_incidence(rp, col, 2, 3)
    g = oracle.Graph(rp, col, 2, 3)
    np.testing.assert_array_equal(inc.s_degree(), g.s_degree())
    kap = g.peel()
    tau, iters = inc.snd()
    np.testing.assert_array_equal(tau, kap)
    assert iters == g.snd()[2]
    for k in (1, 2):
        np.testing.assert_array_equal(inc.iterate_k("snd", k)[0], g.snd(max_sweeps=k)[0])
    t2, _, _ = inc.and_(notify=True)
    np.testing.assert_array_equal(t2, kap)

"""Pins for the CPU oracle: each check ties it to something other than itself.

* values the paper prints (worked examples in tests/golden/),
* closed forms (cliques, cycles, stars, unions, cocktail-party graphs,
  complete bipartite graphs, wheels, windmills, the Petersen graph),
* brute force on tiny graphs (Lemma 1 over all subsets; repeated deletion;
  the SND trace from Def. 4 and the degree levels from Def. 5, written with
  sets),
* theorems (Thm. 1 monotonicity and lower bound, Thm. 3 level-by-level
  convergence, AND never slower than SND),
* library routines (networkx core numbers where installed, scipy's Kendall tau),
* rejection of malformed CSR input.

A plausible slip in the oracle -- a dropped s-clique, max instead of min in
rho, an off-by-one in H, a wrong r-clique id -- fails at least one of these;
test_oracle_mutants.py plants such slips one at a time to show it.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1704_00386_gb300 import graphs as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RS = [(1, 2), (2, 3), (3, 4)]


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _random_graph(rng, n_lo, n_hi, m_hi):
    n = int(rng.integers(n_lo, n_hi + 1))
    e = rng.integers(0, n, size=(int(rng.integers(0, m_hi + 1)), 2))
    return G.to_csr(n, e[:, 0], e[:, 1])


# ---------------------------------------------------------------- h-index

def test_hindex_paper_values():
    for case in _gold("hindex_paper.json")["cases"]:
        assert oracle.hindex(case["K"]) == case["H"], case["where"]


def test_hindex_special_cases():
    assert oracle.hindex([]) == 0                 # empty multiset
    assert oracle.hindex([0, 0, 0]) == 0
    assert oracle.hindex([5]) == 1
    assert oracle.hindex([1, 1, 1, 1]) == 1       # duplicates count
    assert oracle.hindex([4, 4, 4, 4]) == 4
    assert oracle.hindex([100] * 7) == 7          # bounded by the size
    assert oracle.hindex(list(range(1, 11))) == 5


def test_hindex_brute_force_random():
    rng = np.random.default_rng(7)
    for _ in range(300):
        k = list(rng.integers(0, 12, size=int(rng.integers(0, 12))))
        # h qualifies iff at least h values are >= h; take the largest
        best = max(h for h in range(len(k) + 1) if sum(v >= h for v in k) >= h)
        assert oracle.hindex(k) == best


# ---------------------------------------------------------- worked example

def _toy():
    return oracle.Graph(*G.toy_core_graph(), 1, 2)


def test_toy_core_numbers_and_degrees():
    gold = _gold("toy_core_fig5_fig6.json")
    g = _toy()
    assert list(g.s_degree()) == gold["degree"]
    assert list(g.peel()) == gold["core_number"]


def test_toy_snd_trace():
    gold = _gold("toy_core_fig5_fig6.json")
    g = _toy()
    assert list(g.snd(max_sweeps=1)[0]) == gold["snd_tau1"]
    assert list(g.snd(max_sweeps=2)[0]) == gold["snd_tau2"]
    tau, sweeps, updating, evals = g.snd()
    assert list(tau) == gold["core_number"]
    assert updating == gold["snd_updating_iterations"]
    assert sweeps == updating + 1            # tau_3 is computed and unchanged


def test_toy_and_orders():
    gold = _gold("toy_core_fig5_fig6.json")
    names = gold["vertices"]
    g = _toy()
    order = [names.index(v) for v in gold["and_level_order"]]
    tau, _, updating, _ = g.and_(notify=False, order=order)
    assert list(tau) == gold["core_number"]
    assert updating == gold["and_level_order_updating_iterations"]
    tau, _, updating, _ = g.and_(notify=False)
    assert updating == gold["and_abc_order_updating_iterations"]


def test_toy_notification_counts():
    gold = _gold("toy_core_fig5_fig6.json")
    g = _toy()
    tau, sweeps, updating, evals = g.and_(notify=True)
    assert list(tau) == gold["core_number"]
    assert evals == gold["and_notify_computations"]
    assert sweeps == gold["and_notify_iterations"]
    # without notification: the paper's 24 computations in 4 iterations count
    # the initialisation tau_0 = d_s as one pass of 6 computations
    tau, sweeps, updating, evals = g.and_(notify=False)
    n = len(gold["vertices"])
    assert evals + n == gold["and_no_notify_computations_incl_init"]
    assert sweeps + 1 == gold["and_no_notify_iterations_incl_init"]


def test_toy_degree_levels():
    gold = _gold("toy_core_fig5_fig6.json")
    g = _toy()
    k, lv = g.degree_levels()
    assert k == 4
    assert {v: int(lv[i]) for i, v in enumerate(gold["vertices"])} == gold["degree_levels"]


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 9])
def test_complete_graph(k):
    rp, col = G.complete_graph(k)
    for (r, s) in RS:
        if k < s:
            continue
        g = oracle.Graph(rp, col, r, s)
        want = k - r            # each r-clique lies in C(k-r, s-r) = k-r s-cliques
        assert (g.peel() == want).all()
        assert (g.snd()[0] == want).all()
        assert g.snd()[2] == 0  # already converged at tau_0 = d_s
        assert g.num_r == len(list(itertools.combinations(range(k), r)))


@pytest.mark.parametrize("k", [4, 5, 8, 13])
def test_cycle(k):
    rp, col = G.cycle_graph(k)
    assert (oracle.Graph(rp, col, 1, 2).peel() == 2).all()
    assert (oracle.Graph(rp, col, 2, 3).peel() == 0).all()
    assert oracle.Graph(rp, col, 3, 4).num_r == 0


@pytest.mark.parametrize("leaves", [1, 2, 7])
def test_star(leaves):
    rp, col = G.star_graph(leaves)
    assert (oracle.Graph(rp, col, 1, 2).peel() == 1).all()
    assert (oracle.Graph(rp, col, 2, 3).peel() == 0).all()


def _edges_csr(n, pairs):
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    return G.to_csr(n, pairs[:, 0], pairs[:, 1])


@pytest.mark.parametrize("half", [3, 4, 6])
def test_cocktail_party_graph(half):
    # K_n minus a perfect matching (n = 2 half): every r-clique sees the same
    # number of s-cliques, so the whole graph attains d_s and kappa = d_s:
    # core n-2, truss n-4 (common neighbours of u,v: all but u, v and their
    # partners), (3,4) n-6
    n = 2 * half
    pairs = [(u, v) for u in range(n) for v in range(u + 1, n) if v != u + half]
    rp, col = _edges_csr(n, pairs)
    for (r, s), want in zip(RS, (n - 2, n - 4, n - 6)):
        g = oracle.Graph(rp, col, r, s)
        if g.num_r == 0:
            continue
        assert (g.s_degree() == want).all()
        assert (g.peel() == want).all() and (g.snd()[0] == want).all()


@pytest.mark.parametrize("a,b", [(1, 5), (3, 3), (4, 7)])
def test_complete_bipartite(a, b):
    # K_{a,b}: core min(a,b), no triangles
    rp, col = _edges_csr(a + b, [(u, a + v) for u in range(a) for v in range(b)])
    assert (oracle.Graph(rp, col, 1, 2).peel() == min(a, b)).all()
    assert (oracle.Graph(rp, col, 2, 3).peel() == 0).all()
    assert oracle.Graph(rp, col, 3, 4).num_r == 0


@pytest.mark.parametrize("rim", [5, 8, 13])
def test_wheel(rim):
    # hub 0 and a rim cycle: every vertex is in the 3-core and no deeper (rim
    # degree 3); a rim edge lies in one triangle, so the 1-truss (triangle
    # convention) is the deepest; the rim triangles lie in no 4-clique once
    # the rim has 5 or more vertices
    pairs = [(0, i) for i in range(1, rim + 1)] + [(i, i % rim + 1) for i in range(1, rim + 1)]
    rp, col = _edges_csr(rim + 1, pairs)
    assert (oracle.Graph(rp, col, 1, 2).peel() == 3).all()
    g = oracle.Graph(rp, col, 2, 3)
    assert (g.peel() == 1).all() and (g.snd()[0] == 1).all()
    t = oracle.Graph(rp, col, 3, 4)
    assert t.num_r == rim and (t.peel() == 0).all()


@pytest.mark.parametrize("blades", [1, 2, 7])
def test_windmill(blades):
    # triangles sharing one vertex: core 2, every edge in exactly one triangle
    pairs = []
    for i in range(blades):
        a, b = 1 + 2 * i, 2 + 2 * i
        pairs += [(0, a), (0, b), (a, b)]
    rp, col = _edges_csr(2 * blades + 1, pairs)
    assert (oracle.Graph(rp, col, 1, 2).peel() == 2).all()
    g = oracle.Graph(rp, col, 2, 3)
    assert (g.s_degree() == 1).all() and (g.peel() == 1).all()
    t = oracle.Graph(rp, col, 3, 4)
    assert t.num_r == blades and (t.peel() == 0).all()


def test_petersen_graph():
    # 3-regular, triangle-free: core 3 everywhere, truss 0
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    rp, col = _edges_csr(10, outer + spokes + inner)
    assert (oracle.Graph(rp, col, 1, 2).peel() == 3).all()
    assert (oracle.Graph(rp, col, 2, 3).peel() == 0).all()


def test_isolated_vertices_and_empty():
    rp = np.zeros(6, np.int64)
    col = np.zeros(0, np.int32)
    g = oracle.Graph(rp, col, 1, 2)
    assert (g.peel() == 0).all() and (g.snd()[0] == 0).all()
    assert oracle.Graph(rp, col, 2, 3).num_r == 0
    g0 = oracle.Graph(np.zeros(1, np.int64), col, 1, 2)
    assert g0.num_r == 0 and g0.peel().size == 0


def test_disjoint_union_decomposes_independently():
    rng = np.random.default_rng(11)
    parts = [_random_graph(rng, 5, 12, 30) for _ in range(3)]
    rp, col = G.disjoint_union(*parts)
    for (r, s) in RS:
        whole = oracle.Graph(rp, col, r, s)
        kw = whole.peel()
        tw = [tuple(t) for t in whole.r_cliques()]
        got = dict(zip(tw, kw.tolist()))
        off = 0
        for prp, pcol in parts:
            g = oracle.Graph(prp, pcol, r, s)
            for t, k in zip(g.r_cliques(), g.peel()):
                assert got[tuple(int(x) + off for x in t)] == k
            off += prp.size - 1


def test_planted_clique_bounds():
    k = 12
    s1, d1 = G.erdos_renyi(120, 3 / 119, seed=21)
    rng = np.random.default_rng(5)
    vs = rng.choice(120, size=k, replace=False)
    a, b = np.triu_indices(k, 1)
    rp, col = G.to_csr(120, np.concatenate([s1, vs[a]]), np.concatenate([d1, vs[b]]))
    inside = set(int(v) for v in vs)
    for (r, s) in RS:
        g = oracle.Graph(rp, col, r, s)
        kap = g.peel()
        for t, kk in zip(g.r_cliques(), kap):
            if set(int(x) for x in t) <= inside:
                assert kk >= k - r


# ------------------------------------------------------------ brute force

def test_brute_force_lemma1_all_rs():
    rng = np.random.default_rng(3)
    checked = {rs: 0 for rs in RS}
    for rs in RS:
        tries = 0
        while checked[rs] < 25 and tries < 400:
            tries += 1
            rp, col = _random_graph(rng, 3, 8, 20)
            g = oracle.Graph(rp, col, *rs)
            if g.num_r > 13 or (rs != (1, 2) and g.num_r == 0):
                continue
            R, bf = oracle.brute_force_kappa(rp, col, *rs)
            assert [tuple(int(x) for x in t) for t in g.r_cliques()] == R
            assert list(g.peel()) == bf
            assert list(g.snd()[0]) == bf
            assert list(g.and_(notify=True)[0]) == bf
            assert list(g.and_(notify=False)[0]) == bf
            checked[rs] += 1
    assert all(v >= 10 for v in checked.values()), checked


def test_naive_deletion_matches_peeling():
    rng = np.random.default_rng(4)
    for rs in RS:
        for _ in range(8):
            rp, col = _random_graph(rng, 6, 16, 60)
            g = oracle.Graph(rp, col, *rs)
            R, kap = oracle.naive_kappa(rp, col, *rs)
            assert [tuple(int(x) for x in t) for t in g.r_cliques()] == R
            assert list(g.peel()) == kap


def test_s_degree_matches_enumeration():
    rng = np.random.default_rng(5)
    for rs in RS:
        for _ in range(6):
            rp, col = _random_graph(rng, 5, 14, 50)
            g = oracle.Graph(rp, col, *rs)
            R = oracle.enumerate_cliques(rp, col, rs[0])
            S = oracle.enumerate_cliques(rp, col, rs[1])
            want = [sum(set(t) <= set(sc) for sc in S) for t in R]
            assert list(g.s_degree()) == want
            assert g.num_incidences == sum(want)


def _members_by_enumeration(rp, col, r, s):
    """r-cliques (canonical order) and, per s-clique, the ids of its r-cliques,
    from the brute-force clique enumeration."""
    R = oracle.enumerate_cliques(rp, col, r)
    S = oracle.enumerate_cliques(rp, col, s)
    rid = {t: i for i, t in enumerate(R)}
    return R, [[rid[sub] for sub in itertools.combinations(sc, r)] for sc in S]


def _h_by_definition(vals):
    return max(h for h in range(len(vals) + 1) if sum(v >= h for v in vals) >= h)


def test_snd_trace_brute_force():
    """Alg. 2 on tiny graphs, every pass checked: tau_{t+1}(R) is H, over the
    s-cliques S containing R, of the smallest tau_t among the other r-cliques
    of S (Def. 4), every value read from tau_t.  Written with sets and the
    brute-force enumeration, and compared at every t, so an in-place update or
    a dropped member changes some pass."""
    rng = np.random.default_rng(11)
    for rs in RS:
        done = tries = 0
        while done < 12 and tries < 500:
            tries += 1
            rp, col = _random_graph(rng, 5, 11, 36)
            R, members = _members_by_enumeration(rp, col, *rs)
            if not R:
                continue
            g = oracle.Graph(rp, col, *rs)
            of = [[mem for mem in members if i in mem] for i in range(len(R))]
            tau = [len(of[i]) for i in range(len(R))]     # tau_0 = d_s
            t = 0
            while True:
                nxt = [_h_by_definition([min(tau[j] for j in mem if j != i) for mem in of[i]])
                       for i in range(len(R))]
                if nxt == tau:
                    break
                t += 1
                assert list(g.snd(max_sweeps=t)[0]) == nxt, (rs, t)
                tau = nxt
            _, sweeps, updating, _ = g.snd()
            assert updating == t and sweeps == t + 1
            done += 1
        assert done == 12, (rs, done)


def test_degree_levels_brute_force():
    """Def. 5 on tiny graphs with the S-degrees recounted from scratch at each
    level: level i is every surviving r-clique of the smallest S-degree among
    the survivors, counting only s-cliques whose r-cliques all survive; the
    level leaves together."""
    rng = np.random.default_rng(12)
    for rs in RS:
        done = tries = 0
        while done < 12 and tries < 500:
            tries += 1
            rp, col = _random_graph(rng, 5, 11, 36)
            R, members = _members_by_enumeration(rp, col, *rs)
            if not R:
                continue
            alive = set(range(len(R)))
            level = [None] * len(R)
            k = 0
            while alive:
                deg = {i: sum(1 for mem in members if i in mem and all(j in alive for j in mem)) for i in alive}
                low = min(deg.values())
                for i in [i for i in alive if deg[i] == low]:
                    level[i] = k
                    alive.discard(i)
                k += 1
            count, lv = oracle.Graph(rp, col, *rs).degree_levels()
            assert count == k and list(lv) == level, rs
            done += 1
        assert done == 12, (rs, done)


# ---------------------------------------------------------------- theorems

def _medium_graphs():
    out = []
    src, dst = G.chung_lu(400, 2.3, 8.0, seed=31)
    out.append(G.to_csr(400, src, dst))
    i, j = G.erdos_renyi(300, 10 / 299, seed=32)
    out.append(G.to_csr(300, i, j))
    n, s2, d2 = G.rmat(9, 8, seed=33)
    out.append(G.to_csr(n, s2, d2))
    return out


@pytest.mark.parametrize("rs", RS)
def test_theorems_on_medium_graphs(rs):
    rng = np.random.default_rng(9)
    for rp, col in _medium_graphs():
        g = oracle.Graph(rp, col, *rs)
        kap = g.peel()
        ds = g.s_degree()
        tau, sweeps, updating, _ = g.snd()
        assert (tau == kap).all()
        levels, lv = g.degree_levels()
        # Thm. 3 / Lemma 2: level L_i has converged after i sweeps
        assert updating <= max(levels - 1, 0)
        prev = ds
        for t in range(1, updating + 1):
            cur = g.snd(max_sweeps=t)[0]
            assert (cur <= prev).all()                 # Thm. 1, monotone
            assert (cur >= kap).all()                  # Thm. 1, lower bound
            assert (cur[lv <= t] == kap[lv <= t]).all()  # Thm. 3
            prev = cur
        # AND reaches the same fixed point, in no more updating sweeps
        for notify in (False, True):
            ta, _, up_a, _ = g.and_(notify=notify)
            assert (ta == kap).all()
            assert up_a <= updating
        order = rng.permutation(g.num_r)
        assert (g.and_(notify=True, order=order)[0] == kap).all()
        # early-stopped AND is sandwiched: kappa <= tau_AND_k <= tau_SND_k
        for k in (1, 2, 3):
            ta = g.and_(notify=False, max_sweeps=k)[0]
            ts = g.snd(max_sweeps=k)[0]
            assert (kap <= ta).all() and (ta <= ts).all()


@pytest.mark.parametrize("rs", RS)
def test_notification_only_skips_no_op_evaluations(rs):
    """Section 4.3: an r-clique is skipped only when no neighbour dropped to
    a value its (tau-clipped) h-index can see, and an update is not followed
    by re-evaluating itself (its new value is already below the clip), so a
    skipped evaluation would have changed nothing.  In one processing order,
    AND with notification therefore follows AND without it pass for pass:
    the same tau after every pass, the same number of passes, and no more
    evaluations (Table 4 reports the savings)."""
    rng = np.random.default_rng(13)
    for rp, col in _medium_graphs():
        g = oracle.Graph(rp, col, *rs)
        for order in (None, rng.permutation(g.num_r)):
            t_nn, sw_nn, up_nn, ev_nn = g.and_(notify=False, order=order)
            t_n, sw_n, up_n, ev_n = g.and_(notify=True, order=order)
            assert (t_n == t_nn).all() and sw_n == sw_nn and up_n == up_nn
            assert ev_n <= ev_nn
            for k in range(1, up_nn + 1):
                a = g.and_(notify=False, order=order, max_sweeps=k)[0]
                b = g.and_(notify=True, order=order, max_sweeps=k)[0]
                assert (a == b).all(), (rs, k)


def test_resume_from_intermediate_tau():
    rp, col = _medium_graphs()[0]
    g = oracle.Graph(rp, col, 2, 3)
    full = g.snd()[0]
    mid = g.snd(max_sweeps=2)[0]
    assert (g.snd(tau=mid)[0] == full).all()
    assert (g.and_(tau=mid)[0] == full).all()


def test_cross_decomposition_bounds():
    for rp, col in _medium_graphs():
        g1, g2, g3 = (oracle.Graph(rp, col, r, s, incidence=False) for r, s in RS)
        k1, k2, k3 = g1.peel(), g2.peel(), g3.peel()
        e = g2.r_cliques()
        # an edge in a k-truss (k triangles each) sits in a (k+1)-core
        assert (k2 + 1 <= np.minimum(k1[e[:, 0]], k1[e[:, 1]])).all()
        t = g3.r_cliques()
        eid = {tuple(x): i for i, x in enumerate(e.tolist())}
        for tri, kk in zip(t.tolist(), k3):
            a, b, c = tri
            m = min(k2[eid[(a, b)]], k2[eid[(a, c)]], k2[eid[(b, c)]])
            assert kk + 1 <= m


def test_networkx_core_number():
    nx = pytest.importorskip("networkx")
    for rp, col in _medium_graphs():
        n = rp.size - 1
        gx = nx.Graph()
        gx.add_nodes_from(range(n))
        for u in range(n):
            for v in col[rp[u]:rp[u + 1]]:
                gx.add_edge(u, int(v))
        want = nx.core_number(gx)
        got = oracle.Graph(rp, col, 1, 2, incidence=False).peel()
        assert [want[u] for u in range(n)] == got.tolist()


def test_rejects_invalid_csr():
    # Section 2: a simple undirected graph, here as a symmetric CSR with
    # strictly increasing rows and no self-loops
    bad = {
        "not symmetric": ([0, 1, 1], [1]),
        "directed cycle (in- and out-degrees match)": ([0, 1, 2, 3], [1, 2, 0]),
        "self-loop": ([0, 2, 3], [0, 1, 0]),
        "duplicate entry": ([0, 2, 4], [1, 1, 0, 0]),
        "unsorted row": ([0, 2, 4, 6], [2, 1, 0, 2, 0, 1]),
        "column out of range": ([0, 1, 2], [1, 2]),
        "negative column": ([0, 1, 2], [-1, 0]),
        "row_ptr[0] != 0": ([1, 2, 3], [1, 0, 0]),
        "decreasing row_ptr": ([0, 2, 1, 2], [1, 2]),
        "a row past the end of col": ([0, 100, 2], [1, 0]),
        "row_ptr ends before col": ([0, 1, 1], [1, 0]),
    }
    for what, (rp, col) in bad.items():
        for rs in RS:
            with pytest.raises(RuntimeError):
                oracle.Graph(np.array(rp, np.int64), np.array(col, np.int32), *rs)
                pytest.fail(what)
    rp2, col2 = G.toy_core_graph()
    with pytest.raises(RuntimeError):
        oracle.Graph(rp2, col2, 1, 3)        # unsupported (r, s)


# ------------------------------------------------------------- PartialAnd

@pytest.mark.parametrize("rs", RS)
def test_partial_and_pins(rs):
    rng = np.random.default_rng(23)
    for rp, col in _medium_graphs():
        g = oracle.Graph(rp, col, *rs)
        if g.num_r == 0:
            continue
        kap = g.peel()
        ds = g.s_degree()
        everyone = np.ones(g.num_r, bool)
        assert (g.partial_and(everyone)[0] == kap).all()        # P = all: plain AND
        nobody = np.zeros(g.num_r, bool)
        assert (g.partial_and(nobody)[0] == ds).all()           # P = empty: d_s untouched
        small = rng.random(g.num_r) < 0.3
        big = small | (rng.random(g.num_r) < 0.4)
        t_small = g.partial_and(small)[0]
        t_big = g.partial_and(big)[0]
        assert (t_small[~small] == ds[~small]).all()
        assert (kap <= t_big).all() and (t_big <= t_small).all()  # more members, tighter
        # any order, with or without notification, and the synchronous form
        # reach the same fixed point
        order = rng.permutation(g.num_r)
        assert (g.partial_and(small, order=order)[0] == t_small).all()
        assert (g.partial_and(small, notify=False)[0] == t_small).all()
        assert (g.partial_snd(small)[0] == t_small).all()


def test_partial_and_brute_force():
    """PartialAnd (end of Section 4.3) on tiny graphs against its definition:
    the update operator of Def. 4 applied to the members only, non-members
    held at d_s, iterated with sets until nothing changes."""
    rng = np.random.default_rng(29)
    for rs in RS:
        done = tries = 0
        while done < 10 and tries < 500:
            tries += 1
            rp, col = _random_graph(rng, 5, 11, 36)
            R, members = _members_by_enumeration(rp, col, *rs)
            if len(R) < 2:
                continue
            of = [[mem for mem in members if i in mem] for i in range(len(R))]
            mask = rng.random(len(R)) < 0.5
            tau = [len(of[i]) for i in range(len(R))]
            while True:
                nxt = [(_h_by_definition([min(tau[j] for j in mem if j != i) for mem in of[i]])
                        if mask[i] else tau[i]) for i in range(len(R))]
                if nxt == tau:
                    break
                tau = nxt
            g = oracle.Graph(rp, col, *rs)
            assert list(g.partial_and(mask)[0]) == tau, rs
            assert list(g.partial_and(mask, notify=False)[0]) == tau, rs
            done += 1
        assert done == 10, (rs, done)


# ---- Kendall-Tau (Section 5.2, Fig. 7) --------------------------------------

def test_kendall_tau_b_hand_counted():
    # pairs of [1,2,2,3] / [1,3,2,2]: three concordant, one discordant, one tie
    # in x, one tie in y: S = 2, n0 = 6, tau_b = 2 / sqrt(5 * 5)
    t, S, tx, ty = oracle.kendall_tau_b([1, 2, 2, 3], [1, 3, 2, 2])
    assert (S, tx, ty) == (2, 1, 1)
    assert t == pytest.approx(0.4, abs=1e-15)


def test_kendall_tau_b_closed_forms_and_symmetries():
    x = np.arange(40)
    assert oracle.kendall_tau_b(x, x)[0] == pytest.approx(1.0)
    assert oracle.kendall_tau_b(x, x[::-1])[0] == pytest.approx(-1.0)
    assert np.isnan(oracle.kendall_tau_b(np.zeros(5), x[:5])[0])  # constant: undefined
    rng = np.random.default_rng(7)
    a = rng.integers(0, 9, 300)
    b = a // 3 + rng.integers(0, 4, 300)
    t = oracle.kendall_tau_b(a, b)[0]
    assert oracle.kendall_tau_b(b, a)[0] == pytest.approx(t, abs=1e-15)
    assert oracle.kendall_tau_b(a, -b)[0] == pytest.approx(-t, abs=1e-15)
    assert oracle.kendall_tau_b(3 * a + 5, b)[0] == pytest.approx(t, abs=1e-15)  # order only


def test_kendall_tau_b_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(8)
    for n, hi in ((60, 3), (500, 12), (3000, 200)):
        a = rng.integers(0, hi, n)
        b = (a + rng.integers(0, hi, n)) // 2
        want = stats.kendalltau(a, b).statistic  # tau-b, the default variant
        assert oracle.kendall_tau_b(a, b)[0] == pytest.approx(want, abs=1e-12)

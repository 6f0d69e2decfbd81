"""Input validation of nd_build_incidence against a plain check, on graphs
one edit away from valid.

The library decides symmetry by searching, for each pair of entries, only
one of the two rows (the shorter one by degree class, floor(log2 of the row
length), then id), and by counting the searching entries.  The edits below are made so that each
side of that rule is hit: an entry removed from the longer or the shorter
row, an entry moved to another target with the row lengths unchanged, an
entry added, and rows of equal length (where the id breaks the tie).  The
plain check is the definition of Section 2 written with Python sets: simple
(no loop, no repeated neighbour, rows sorted) and symmetric.  Every edited
graph must be refused with ND_E_INVAL exactly when the plain check refuses
it, for all three (r, s).
"""
import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RS = [(1, 2), (2, 3), (3, 4)]


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd as _nd
    return _nd


def _lists(rp, col):
    return [list(col[rp[u]:rp[u + 1]]) for u in range(len(rp) - 1)]


def _csr(lists):
    rp = np.concatenate([[0], np.cumsum([len(l) for l in lists])]).astype(np.int64)
    col = np.array([v for l in lists for v in l], np.int32)
    return rp, col


def _plain_ok(lists):
    n = len(lists)
    for u, l in enumerate(lists):
        if any(not (0 <= v < n) or v == u for v in l) or any(a >= b for a, b in zip(l, l[1:])):
            return False
    sets = [set(l) for l in lists]
    return all(u in sets[v] for u in range(n) for v in sets[u])


def _edits(lists, rng):
    """(name, edited lists) pairs, each one edit away from `lists`: for each
    of a few entries (u, v), (u, v) dropped, moved to a target w not in row
    u, and (u, w) added.  The entries include one from the longest row to a
    shorter one and one from a shorter row to a longer one."""
    n = len(lists)
    key = [(len(l), u) for u, l in enumerate(lists)]
    hub = max(range(n), key=lambda u: key[u])
    down = (hub, min(lists[hub], key=lambda v: key[v]))            # from the longer row
    leaf = min((u for u in range(n) if lists[u]), key=lambda u: key[u])
    up = (leaf, max(lists[leaf], key=lambda v: key[v]))            # from the shorter row
    picks = [down, up]
    nz = [u for u in range(n) if lists[u]]
    for _ in range(4):
        u = int(rng.choice(nz))
        picks.append((u, int(rng.choice(lists[u]))))
    out = []
    for u, v in picks:
        side = "longer" if key[u] > key[v] else "shorter"
        ed = [list(l) for l in lists]
        ed[u].remove(v)
        out.append(("drop (%d,%d) from the %s row" % (u, v, side), ed))
        cand = [w for w in range(n) if w != u and w not in lists[u]]
        if cand:
            w = int(rng.choice(cand))
            ed = [list(l) for l in lists]
            ed[u].remove(v)
            ed[u] = sorted(ed[u] + [w])
            out.append(("move (%d,%d) to (%d,%d)" % (u, v, u, w), ed))
            ed = [list(l) for l in lists]
            ed[u] = sorted(ed[u] + [w])
            out.append(("add (%d,%d)" % (u, w), ed))
    return out


def _check(nd, lists):
    rp, col = _csr(lists)
    want_ok = _plain_ok(lists)
    for r, s in RS:
        if want_ok:
            inc = nd.build_incidence(rp, col, r, s)
            inc.free()
        else:
            with pytest.raises(nd.NDError) as e:
                nd.build_incidence(rp, col, r, s)
            assert e.value.status == nd.ND_E_INVAL
    return want_ok


@pytest.mark.parametrize("seed", range(4))
def test_one_edit_from_valid_power_law(nd, seed):
    n = 120 + 37 * seed
    s, d = G.chung_lu(n, 2.1, 6.0, seed=500 + seed)
    rp, col = G.to_csr(n, s, d)
    lists = _lists(rp, col)
    assert _check(nd, lists)
    rng = np.random.default_rng(900 + seed)
    for name, ed in _edits(lists, rng):
        assert not _check(nd, ed), name


def test_one_edit_from_valid_equal_row_lengths(nd):
    """A cycle with chords at fixed stride: every row has length 4 (one
    degree class), so the id alone decides which entry of each pair
    searches."""
    n = 64
    lists = [sorted({(u + 1) % n, (u - 1) % n, (u + 9) % n, (u - 9) % n}) for u in range(n)]
    assert _check(nd, lists)
    rng = np.random.default_rng(77)
    for name, ed in _edits(lists, rng):
        assert not _check(nd, ed), name
    # every row length unchanged: (0,1) -> (0,2) and (2,3) -> (2,0) leave
    # (1,0) and (3,2) without their reverses
    ed = [list(l) for l in lists]
    ed[0] = sorted((set(ed[0]) - {1}) | {2})
    ed[2] = sorted((set(ed[2]) - {3}) | {0})
    assert [len(l) for l in ed] == [4] * n
    assert not _check(nd, ed)


def test_one_edit_from_valid_long_rows(nd):
    """A hub of 5,000 leaves (its row is validated in segments), the leaves
    on a path: removing a hub entry, a leaf entry, or moving a leaf's hub
    entry to another leaf must each be refused."""
    n = 5001
    lists = [list(range(1, n))] + [[0] for _ in range(1, n)]
    for leaf in range(1, n - 1):
        lists[leaf].append(leaf + 1)
        lists[leaf + 1].append(leaf)
    lists = [sorted(l) for l in lists]
    rp, col = _csr(lists)
    for r, s in RS:
        nd.build_incidence(rp, col, r, s).free()
    cases = []
    ed = [list(l) for l in lists]
    ed[0].remove(2500)
    cases.append(ed)
    ed = [list(l) for l in lists]
    ed[2500].remove(0)
    cases.append(ed)
    ed = [list(l) for l in lists]
    ed[2500] = sorted((set(ed[2500]) - {0}) | {4000})
    cases.append(ed)
    for ed in cases:
        rp, col = _csr(ed)
        for r, s in RS:
            with pytest.raises(nd.NDError) as e:
                nd.build_incidence(rp, col, r, s)
            assert e.value.status == nd.ND_E_INVAL

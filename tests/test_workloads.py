"""The seeded synthetic workloads: the sizes the design document states, and
the same arrays on every call (the seeds fix them).  CPU only."""
import numpy as np

from paper_1704_00386_gb300 import graphs as G


def _simple(rp, col):
    n = rp.size - 1
    for u in range(0, n, max(1, n // 50)):
        row = col[rp[u]:rp[u + 1]]
        assert (np.diff(row) > 0).all() and not (row == u).any()
    deg = np.diff(rp)
    u = np.repeat(np.arange(n), deg)
    fwd = set(zip(u.tolist()[:5000], col.tolist()[:5000]))
    full = set(zip(u.tolist(), col.tolist()))
    assert all((v, x) in full for x, v in fwd)  # symmetric (sampled)


def test_chunglu_2000_core_workload():
    w = G.workload("chunglu_n2000_g2.5_d10")
    assert (w["r"], w["s"]) == (1, 2)
    assert w["row_ptr"].size - 1 == 2000 and w["col"].size // 2 == 9753
    _simple(w["row_ptr"], w["col"])
    w2 = G.workload("chunglu_n2000_g2.5_d10")
    assert np.array_equal(w["col"], w2["col"]) and np.array_equal(w["row_ptr"], w2["row_ptr"])


def test_chunglu_100000_planted_nucleus_workload():
    w = G.workload("chunglu_n100000_g2.1_d20_planted200")
    assert (w["r"], w["s"]) == (3, 4)
    assert w["row_ptr"].size - 1 == 100000 and w["col"].size // 2 == 1140801
    _simple(w["row_ptr"], w["col"])


def test_rmat_truss_workload_shape():
    w = G.workload("rmat_s16_ef16")
    assert (w["r"], w["s"]) == (2, 3)
    assert w["row_ptr"].size - 1 == 1 << 16 and w["col"].size // 2 == 910000
    _simple(w["row_ptr"], w["col"])


def test_degree_class_numbering_is_a_renumbering():
    # the _byclass truss workload is the same graph with new vertex ids
    w0 = G.workload("rmat_s12_ef16")
    rp, col = w0["row_ptr"], w0["col"]
    w = G.workload("rmat_s12_ef16_byclass")
    rp2, col2 = w["row_ptr"], w["col"]
    _simple(rp2, col2)
    _, _, new_of_old = G.number_by_degree_class(rp, col)
    n = rp.size - 1
    assert sorted(new_of_old.tolist()) == list(range(n))
    src = np.repeat(np.arange(n), np.diff(rp))
    mapped = set(zip(new_of_old[src].tolist(), new_of_old[col].tolist()))
    src2 = np.repeat(np.arange(n), np.diff(rp2))
    assert mapped == set(zip(src2.tolist(), col2.tolist()))
    # degree classes never increase along the new ids; isolated vertices last
    deg2 = np.diff(rp2)
    cls = np.where(deg2 > 0, np.floor(np.log2(np.maximum(deg2, 1))) + 1, 0)
    assert (np.diff(cls) <= 0).all()

"""The multi-threaded SND that times the CPU baseline (oracle/snd_mt.c),
pinned against the single-threaded oracle: the same incidence size and the
same tau after every pass (SND iterates are deterministic, Alg. 2), on one
thread and on several, and the same fixed point kappa as the oracle's
peeling (Thm. 3)."""
import numpy as np
import pytest

import oracle
from paper_1704_00386_gb300 import graphs as G


def _graphs():
    s1, d1 = G.chung_lu(400, 2.3, 9.0, seed=5)
    s2, d2 = G.plant_cliques(400, 3, 8, 16, seed=6)
    yield G.to_csr(400, np.concatenate([s1, s2]), np.concatenate([d1, d2]))
    n, s, d = G.rmat(10, 16, seed=7)
    yield G.to_csr(n, s, d)
    yield G.hub_graph(3000, 6, seed=107)
    yield G.to_csr(5, np.zeros(0, np.int64), np.zeros(0, np.int64))   # no edges at all


@pytest.mark.parametrize("r", [1, 2])
def test_parallel_snd_follows_the_oracle_pass_by_pass(r):
    for rp, col in _graphs():
        ref = oracle.Graph(rp, col, r, r + 1, incidence=True)
        kappa = oracle.decompose(rp, col, r, r + 1)
        for threads in (1, 4):
            par = oracle.ParallelSND(rp, col, r, threads=threads)
            assert par.num_r == ref.num_r
            assert par.num_incidences == ref.num_incidences
            for k in (1, 2, 3):
                want = ref.snd(max_sweeps=k)
                got = par.snd(max_sweeps=k)
                np.testing.assert_array_equal(got[0], want[0])
                assert got[1:] == want[1:]
            want = ref.snd()
            got = par.snd()
            np.testing.assert_array_equal(got[0], kappa)
            assert got[1:] == want[1:]
            # resuming from an iterate continues the same trajectory
            t2 = par.snd(max_sweeps=2)[0]
            np.testing.assert_array_equal(par.snd(tau=t2, max_sweeps=1)[0], ref.snd(max_sweeps=3)[0])


def test_parallel_snd_rejects_what_the_oracle_rejects():
    rp = np.array([0, 1, 1], np.int64)
    col = np.array([1], np.int32)        # 0 -> 1 without 1 -> 0: not symmetric
    with pytest.raises(RuntimeError):
        oracle.ParallelSND(rp, col, 2)
    with pytest.raises(RuntimeError):
        oracle.ParallelSND(*G.complete_graph(5), 3)   # (3,4) is not offered here

"""Serving loop: requests that arrive while others run are admitted as
memory and workers free up, run concurrently on separate streams (and in
disjoint-union batches), and every result equals the result computed alone."""
import threading
import time

import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(17)
    reqs = []
    jobs = [(1, 2), (2, 3), (3, 4)]
    modes = ["snd", "and", "and_nn"]
    for i, (rp, col, _) in enumerate(G.batch_graphs(30, seed=21, n_lo=50, n_hi=4000)):
        job = (1, 2) if i < 8 else jobs[i % 3]      # the opening burst is mostly one job
        mode = "and" if i < 8 else modes[int(rng.integers(0, 3))]
        reqs.append((rp, col, *job, mode))
    reqs.append((*G.hub_graph(3000, 6, seed=107), 2, 3, "and"))
    w = G.workload("chunglu_n2000_g2.5_d10")
    reqs.append((w["row_ptr"], w["col"], 1, 2, "snd"))
    return reqs


def test_results_alone_equal_results_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd, serve
    reqs = _requests()
    alone = []
    for rp, col, r, s, mode in reqs:
        inc = nd.build_incidence(rp, col, r, s)
        if mode == "snd":
            alone.append(inc.snd()[0])
        else:
            alone.append(inc.and_(notify=(mode == "and"))[0])
        inc.free()
    srv = serve.Server(budget_bytes=4 << 30, workers=2, batch_bytes=256 << 20)
    handles = []
    # a burst at t = 0 (more requests than workers: some must wait and be
    # batched together), then Poisson arrivals while earlier ones still run
    burst = 12
    arrivals = np.concatenate([np.zeros(burst), serve.poisson_arrivals(400.0, len(reqs) - burst, seed=3)])
    t0 = time.perf_counter()

    def client():
        for (rp, col, r, s, mode), at in zip(reqs, arrivals):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            handles.append(srv.submit(rp, col, r, s, mode))

    th = threading.Thread(target=client)
    th.start()
    th.join()
    srv.close()
    assert len(handles) == len(reqs)
    batched = 0
    for h, want in zip(handles, alone):
        assert h.done.is_set() and h.error is None, h.error
        np.testing.assert_array_equal(h.result, want)
        batched += h.batched_with > 1
    stats = serve.latency_stats(handles)
    assert stats["count"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"]
    assert batched > 0  # some requests shared a batch


def test_admission_rejects_oversized_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import serve
    srv = serve.Server(budget_bytes=1 << 20, workers=1)
    rp, col = G.complete_graph(60)
    h = srv.submit(rp, col, 3, 4)
    srv.close()
    assert h.error is not None and "budget" in h.error

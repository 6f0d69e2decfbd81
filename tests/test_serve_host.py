"""The serving loop's host logic, without a GPU: footprint bounds and the
admission / grouping rule of Server._take (oldest admissible request first,
then every waiting request of the same job and mode under the byte cap and
the budget, in arrival order)."""
import threading

import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G
from paper_1704_00386_gb300.serve import Request, Server, footprint_bytes


def _bare_server(budget, batch_bytes=1 << 30, max_batch=64, max_wait_s=1e9):
    srv = Server.__new__(Server)  # no workers, no device
    srv.budget, srv.batch_bytes, srv.max_batch, srv.max_wait_s = budget, batch_bytes, max_batch, max_wait_s
    srv.used, srv.queue, srv.cv, srv.closing, srv.next_id, srv.completed = 0, [], threading.Condition(), False, 0, []
    return srv


def _req(r, s, mode, fp, rid):
    q = Request(np.zeros(1, np.int64), np.zeros(0, np.int32), r, s, mode)
    q.footprint, q.rid = fp, rid
    return q


def test_footprint_bounds_the_incidence():
    rp, col = G.complete_graph(12)
    f1, f2, f3 = (footprint_bytes(rp, col, r) for r in (1, 2, 3))
    # K12: 66 edges in 10 triangles each, 220 triangles in 9 four-cliques each
    # (2,3): two 8-byte incidence buffers at the build's peak
    assert f2 >= 2 * 8 * 66 * 10 + (1 << 20) and f3 >= 12 * 220 * 9 + (1 << 20)
    assert f1 < f2 < f3
    big_rp, big_col = G.complete_graph(40)
    assert footprint_bytes(big_rp, big_col, 2) > f2


def test_take_groups_one_job_in_arrival_order_under_the_caps():
    srv = _bare_server(budget=1000, batch_bytes=300, max_batch=3)
    srv.queue = [_req(2, 3, "and", 100, 0), _req(1, 2, "and", 100, 1), _req(2, 3, "and", 100, 2),
                 _req(2, 3, "snd", 100, 3), _req(2, 3, "and", 100, 4), _req(2, 3, "and", 100, 5)]
    group = srv._take()
    assert [g.rid for g in group] == [0, 2, 4]          # same job and mode; cap of 300 bytes
    assert srv.used == 300 and [q.rid for q in srv.queue] == [1, 3, 5]
    assert [g.rid for g in srv._take()] == [1]           # next oldest, a different job
    assert srv.used == 400


def test_take_skips_what_does_not_fit_the_budget():
    srv = _bare_server(budget=250)
    srv.used = 100
    srv.queue = [_req(2, 3, "and", 200, 0), _req(1, 2, "and", 100, 1)]
    assert [g.rid for g in srv._take()] == [1]           # the oldest waits for room
    assert srv._take() == []                             # nothing else fits
    srv.used = 0
    assert [g.rid for g in srv._take()] == [0]


def test_submit_rejects_a_request_larger_than_the_budget():
    srv = _bare_server(budget=1 << 10)
    rp, col = G.complete_graph(30)
    req = srv.submit(rp, col, 3, 4)
    assert req.done.is_set() and "budget" in req.error and srv.queue == []


def test_aging_stops_small_requests_from_starving_a_large_one():
    """Once the oldest request has waited past max_wait_s and still does not
    fit, later requests are held back until it does."""
    srv = _bare_server(budget=1000, max_wait_s=0.5)
    srv.used = 600
    big = _req(2, 3, "and", 800, 0)
    big.arrival = 10.0
    small = [_req(1, 2, "and", 100, i) for i in range(1, 4)]
    for q in small:
        q.arrival = 10.1
    srv.queue = [big] + small
    assert [g.rid for g in srv._take(now=10.2)] == [1, 2, 3]  # still young: the small ones go ahead
    assert srv.used == 900
    srv.queue.extend(_req(1, 2, "and", 100, i) for i in range(4, 6))
    for q in srv.queue[1:]:
        q.arrival = 10.9
    srv.used = 600
    assert srv._take(now=11.0) == []                         # the big one is old: reserve for it
    srv.used = 200                                           # running work finishes
    assert [g.rid for g in srv._take(now=11.1)] == [0]       # it fits now and goes first
    assert [g.rid for g in srv._take(now=11.1)] == []        # nothing else fits next to it
    srv.used = 0
    assert [g.rid for g in srv._take(now=11.2)] == [4, 5]


def test_cancel_withdraws_a_waiting_request_only():
    srv = _bare_server(budget=1000)
    a, b = _req(2, 3, "and", 100, 0), _req(2, 3, "and", 100, 1)
    srv.queue = [a, b]
    assert srv.cancel(a) is True
    assert a.done.is_set() and a.error == "cancelled" and srv.queue == [b]
    assert srv.cancel(a) is False                            # not waiting any more
    taken = srv._take()
    assert taken == [b]
    assert srv.cancel(b) is False                            # a worker has it: it runs to completion
    assert not b.done.is_set() and b.error is None

"""Failure paths that are made on the host, with no GPU fault: a host-side
wait that runs out (ND_E_TIMEOUT), a second call on a handle in use
(ND_E_BUSY), and a per-handle memory limit (ND_E_NOMEM).

The stream is held by torch.cuda._sleep, a kernel that spins for a fixed
number of clock cycles (about a second here) and then ends by itself; the
library's wait is set shorter than that.  After each failure the stream is
drained and the same handle must give the oracle's kappa again.
"""
import threading
import time

import numpy as np
import pytest

from paper_1704_00386_gb300 import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SLEEP_CYCLES = 2_000_000_000   # ~1 s at 2 GHz; it ends by itself


def _nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00386_gb300 import nd
    return nd


def _graph():
    s1, d1 = G.chung_lu(3000, 2.3, 10.0, seed=71)
    s2, d2 = G.plant_cliques(3000, 4, 10, 20, seed=72)
    return G.to_csr(3000, np.concatenate([s1, s2]), np.concatenate([d1, d2]))


def test_wait_limit_gives_timeout_and_the_handle_recovers():
    import oracle
    nd = _nd()
    rp, col = _graph()
    want = oracle.decompose(rp, col, 2, 3)
    inc = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), 2, 3)
    torch.cuda.synchronize()
    try:
        nd.set_wait_limit(0.1)
        torch.cuda._sleep(SLEEP_CYCLES)          # holds the stream for about a second
        with pytest.raises(nd.NDError) as e:
            inc.snd()
        assert e.value.status == nd.ND_E_TIMEOUT
        assert "did not finish within 0.1 s" in str(e.value)
    finally:
        nd.set_wait_limit(600.0)
    torch.cuda.synchronize()                     # the enqueued passes finish; nothing is left hanging
    got, _ = inc.snd()
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    got_and, _, _ = inc.and_(notify=True)
    np.testing.assert_array_equal(got_and.cpu().numpy(), want)
    inc.free()


def test_second_call_on_a_busy_handle_is_refused():
    import oracle
    nd = _nd()
    rp, col = _graph()
    want = oracle.decompose(rp, col, 2, 3)
    inc = nd.build_incidence(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), 2, 3)
    torch.cuda.synchronize()
    first = {}

    def run():
        try:
            first["tau"] = inc.snd()[0]
        except Exception as exc:  # reported below
            first["err"] = exc

    torch.cuda._sleep(SLEEP_CYCLES)              # the first call waits behind this
    t = threading.Thread(target=run)
    t.start()
    time.sleep(0.3)                              # the first call now holds the handle
    with pytest.raises(nd.NDError) as e:
        inc.snd()
    assert e.value.status == nd.ND_E_BUSY
    with pytest.raises(nd.NDError) as e:
        inc.last_passes()
    assert e.value.status == nd.ND_E_BUSY
    t.join(timeout=120)
    assert not t.is_alive() and "err" not in first, first.get("err")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(first["tau"].cpu().numpy(), want)
    got, _ = inc.snd()                           # free again
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    inc.free()


def test_handle_memory_limit_refuses_the_build():
    import oracle
    nd = _nd()
    rp, col = _graph()
    rp_d, col_d = torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()
    try:
        nd.set_handle_memory_limit(64 << 10)     # 64 KB: below even the k-core handle (CSR copy 150 KB)
        for r, s in ((1, 2), (2, 3), (3, 4)):
            with pytest.raises(nd.NDError) as e:
                nd.build_incidence(rp_d, col_d, r, s)
            assert e.value.status == nd.ND_E_NOMEM
            assert "limit" in str(e.value)
    finally:
        nd.set_handle_memory_limit(0)
    for r, s in ((1, 2), (2, 3), (3, 4)):
        inc = nd.build_incidence(rp_d, col_d, r, s)
        bytes_held = inc.incidence_bytes()
        got, _ = inc.snd()
        inc.free()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.decompose(rp, col, r, s))
        # a limit just above what the handle holds after its build lets the build through
        try:
            nd.set_handle_memory_limit(bytes_held + (64 << 20))
            inc = nd.build_incidence(rp_d, col_d, r, s)
            got, _ = inc.snd()
            inc.free()
        finally:
            nd.set_handle_memory_limit(0)
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.decompose(rp, col, r, s))

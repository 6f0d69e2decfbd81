"""The replicas path of bench.py on CPU ranks (gloo, world size 2): the
whole-job rate is the units of all ranks over the slowest rank's time, and
the reference arm runs on rank 0 alone.  No GPU involved."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 150.0][rank]
    units = [1000.0, 3000.0][rank]
    rate, ms_max, total = bench.job_rate(ms, units, dist, "cpu")
    single = bench.job_rate(ms, units)
    args = bench.argparse.Namespace(warmup=0, steps=0, gpus=world, workload="w")
    ref_rc = bench.run_reference(args, 1, world) if rank == 1 else 0  # non-zero ranks do no work
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, rate, ms_max, total, single, ref_rc))


def test_job_rate_over_two_gloo_ranks():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max, total, single, ref_rc in res:
        assert ms_max == 150.0 and total == 4000.0
        assert rate == pytest.approx(4000.0 / 0.150)
        assert single[0] == pytest.approx([1000.0 / 0.100, 3000.0 / 0.150][rank])
        assert ref_rc == 0

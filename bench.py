#!/usr/bin/env python
"""Benchmark: r-clique h-index updates/sec to convergence on GB300.

Workload (default): k-truss, (r,s) = (2,3), of an R-MAT graph, scale 20,
edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05), seed 2, symmetrised,
deduplicated, no self-loops (15.7M edges, 424M triangles).

One step = the whole hot path on one graph, inputs resident in HBM:
incidence build (validation, canonical edge ids, triangle count, scan,
triangle fill, degree buckets), SND to convergence, AND with notification
to convergence, results in device buffers, incidence freed.
value = h-index evaluations (SND + AND) / device time of the steps.

--gpus N: N independent replicas, one per GPU (the method has no exchange
step; each rank decomposes its own copy), launched by torchrun; value is the
evaluations of all ranks / the slowest rank's time.

--impl reference: the CPU oracle (plain single-threaded C) on a bounded
sample of the same workload (R-MAT scale 14, same generator), rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "r-clique h-index updates/sec to convergence; HBM GB/s vs peak; batched p99"
UNIT = "updates/s"
CPU_SAMPLE_SCALE = 14


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="rmat_s20_ef16")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# --------------------------------------------------------------------- utils

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def cpu_oracle_sample(scale: int = CPU_SAMPLE_SCALE):
    """The oracle's whole path (its own incidence build, SND, AND with
    notification) on R-MAT scale `scale`, single-threaded."""
    import oracle
    from paper_1704_00386_gb300 import graphs as G
    n, s, d = G.rmat(scale, 16, seed=2)
    rp, col = G.to_csr(n, s, d)
    t0 = time.perf_counter()
    g = oracle.Graph(rp, col, 2, 3, incidence=True)
    _, sw, _, ev_s = g.snd()
    _, _, _, ev_a = g.and_(notify=True)
    dt = time.perf_counter() - t0
    return (ev_s + ev_a) / dt, dt, ev_s + ev_a, f"R-MAT scale {scale} EF16 (2,3), oracle build+SND+AND"


# ----------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    rates, times = [], []
    sample = ""
    for i in range(args.warmup + args.steps):
        rate, dt, ev, sample = cpu_oracle_sample()
        if i >= args.warmup:
            rates.append(rate)
            times.append(dt)
    total_ev_rate = sum(r * t for r, t in zip(rates, times)) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": total_ev_rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample},
        "cpu_baseline": {"value": total_ev_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": total_ev_rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    nd.load(build_if_missing=False)

    w = G.workload(args.workload)
    r, s = w["r"], w["s"]
    rp_h, col_h = w["row_ptr"], w["col"]
    rp_d = torch.from_numpy(rp_h).to(dev)
    col_d = torch.from_numpy(col_h).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def one_step():
        inc = nd.build_incidence(rp_d, col_d, r, s)
        tau_s, it_s = inc.snd()
        _, ev = inc.last_passes()
        ev_s = int(ev.sum())
        tau_a, it_a, ev_a = inc.and_(notify=True)
        info = dict(num_r=inc.num_r, M=inc.num_incidences, q=inc.q, snd_iters=it_s,
                    and_iters=it_a, snd_evals=ev_s, and_evals=ev_a)
        inc.free()
        return tau_s, tau_a, info

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one_step()
    barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    nd.prof_enable(True)
    step_ms, infos = [], []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        tau_s, tau_a, info = one_step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        infos.append(info)
    barrier()
    prof = nd.prof_read()
    nd.prof_enable(False)
    clk = clocks.stop()

    total_ms = sum(step_ms)
    evals_rank = sum(i["snd_evals"] + i["and_evals"] for i in infos)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms_max = float(t.item())
        e = torch.tensor([evals_rank], dtype=torch.float64, device=dev)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        evals_all = float(e.item())
    else:
        total_ms_max, evals_all = total_ms, float(evals_rank)
    value = evals_all / (total_ms_max / 1000.0)

    # parity of the timed results (bit-exact against the oracle's digest)
    tau_host = tau_s.cpu().numpy()
    same = bool(torch.equal(tau_s, tau_a))
    parity = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "digests.json")) as f:
            gold = json.load(f).get(args.workload)
        if gold:
            parity = (sha(tau_host) == gold["kappa_sha256"]) and same
    except FileNotFoundError:
        pass

    # ----- roofline of the dominant kernel
    info = infos[-1]
    peak, peak_kind = load_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, ms) = top
    N_R, M, q = info["num_r"], info["M"], info["q"]
    if name == "snd_pass":
        eff = sum(i["snd_iters"] + 1 for i in infos)
        per_launch = 4.0 * q * M + 24.0 * N_R
        units = f"{q}*4 B ids per incidence x {M} + 24 B x {N_R} r-cliques, per effective pass"
    elif name in ("tri_fill", "tri_count"):
        eff = launches
        per_launch = (8.0 * M if name == "tri_fill" else 0.0) + 4.0 * (rp_h[-1]) + 8.0 * (rp_h.size) + 16.0 * N_R
        units = "CSR read + edge arrays + 8 B per incidence written (fill)"
    else:
        eff = launches
        per_launch = 4.0 * q * M + 24.0 * N_R
        units = "4q B per incidence + 24 B per r-clique"
    avg_ms = ms / max(eff, 1)
    achieved = per_launch / (avg_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "bytes_per_launch": per_launch, "launches_effective": eff, "avg_launch_ms": avg_ms,
                "units": units}

    # ----- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        rp_pin = torch.from_numpy(rp_h).pin_memory().numpy()
        col_pin = torch.from_numpy(col_h).pin_memory().numpy()
        out_s = torch.empty(N_R, dtype=torch.int32).pin_memory().numpy()
        out_a = torch.empty(N_R, dtype=torch.int32).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        ev_total = 0
        for _ in range(args.steps):
            inc = nd.build_incidence(rp_pin, col_pin, r, s)
            _, _ = inc.snd(out=out_s)
            _, ev = inc.last_passes()
            _, _, ev_a = inc.and_(notify=True, out=out_a)
            ev_total += int(ev.sum()) + ev_a
            inc.free()
        barrier()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
            e = torch.tensor([float(ev_total)], dtype=torch.float64, device=dev)
            dist.all_reduce(e, op=dist.ReduceOp.SUM)
            ev_total = float(e.item())
        e2e = {"value": ev_total / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(rp_pin.nbytes + col_pin.nbytes),
               "d2h_bytes_per_step": int(out_s.nbytes + out_a.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, ev, sample = cpu_oracle_sample()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "seconds": dt}

    if rank == 0:
        phases = {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "recipe": w["recipe"], "r": r, "s": s,
                       "n": int(rp_h.size - 1), "edges": int(rp_h[-1] // 2), "r_cliques": N_R,
                       "incidences": M, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "gpu_launches": int(sum(v[0] for v in prof.values())),
            "clocks": clk,
            "per_step": {"snd_iters": info["snd_iters"], "and_iters": info["and_iters"],
                         "snd_evals": info["snd_evals"], "and_evals": info["and_evals"],
                         "step_ms": step_ms},
            "kernels": phases,
            "parity_vs_oracle_digest": parity, "snd_equals_and": same,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    rc = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())

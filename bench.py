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

--impl reference: the CPU oracle on the same graph, rank 0 only: its SND
(Alg. 2, the oracle's arithmetic) with the loop over r-cliques split over
every host core, one full pass per step, the incidence built once before
the timed steps.

After the timed region the default run also measures, without touching the
headline: SND, AND and AND-nn side by side on the three single-graph
workloads (Chung-Lu 2,000-vertex k-core, R-MAT scale-20 k-truss, Chung-Lu
100,000-vertex (3,4) with planted cliques), the R-MAT scale-26 k-core (one step), 256 graphs of the batched workload (one
disjoint-union batch, autotuned, against one graph per launch) and a short
Poisson request stream (p50 / p99), under "extra".
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
PEEL_SAMPLE_SCALE = 14    # the single-threaded peeling oracle, timed on a bounded sample
CPU_SND_SECONDS = 10.0    # time budget of the multi-threaded SND passes of the CPU baseline
# ncu DRAM bytes per incidence of the SND pass (k-truss, q = 2), measured on the
# current kernels on R-MAT scale 18: pass 12, with the rho cache (dram__bytes_read.sum +
# dram__bytes_write.sum = 2.197118 GB + 32.99328 MB per pass over 247,767,033
# incidences, 9.00 B), and pass 21 of the late-pass kernel without it (2.195024 GB +
# 26.116608 MB, 8.96 B); None once a kernel changes until it is measured again.
NCU_SND_TRAFFIC_PER_INCIDENCE = (2.197118e9 + 32.99328e6) / 247767033


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="rmat_s20_ef16")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mode", choices=["single", "batch", "serve", "otf", "quality", "noalloc", "sweeps"],
                   default="single",
                   help="single: one graph per step (default); batch: many graphs as one disjoint "
                        "union vs one graph per launch; serve: Poisson request stream, p50/p99; "
                        "otf: stored incidence vs no-storage passes; quality: Kendall-Tau and "
                        "accuracy of the early-stopped iterates against kappa; noalloc: the "
                        "allocation-free k-core entry point against build + SND; sweeps: SND, AND "
                        "and AND-nn to convergence on the Chung-Lu 2K k-core, R-MAT s20 k-truss and "
                        "Chung-Lu 100K (3,4) workloads (or --workload)")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--requests", type=int, default=192)
    p.add_argument("--no-extras", action="store_true",
                   help="skip the measurements after the timed region (scale-26 k-core, batch, serve)")
    p.add_argument("--cpu-threads", type=int, default=0, help="threads of the CPU baseline (0 = all)")
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


def workload_config(w, rp_h, num_r=None, incidences=None, world=1):
    """The config block both arms print for the same workload."""
    cfg = {"workload": w["name"], "recipe": w["recipe"], "r": w["r"], "s": w["s"],
           "n": int(rp_h.size - 1), "edges": int(rp_h[-1] // 2),
           "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"}
    if num_r is not None:
        cfg["r_cliques"] = int(num_r)
    if incidences is not None:
        cfg["incidences"] = int(incidences)
    return cfg


class CpuSND:
    """The oracle's SND on all host cores (oracle.ParallelSND: Alg. 2 with the
    loop over r-cliques split over threads), on the graph of the workload
    itself.  The incidence is built once (its seconds are reported)."""

    def __init__(self, rp, col, r, threads=0):
        import oracle
        t0 = time.perf_counter()
        self.g = oracle.ParallelSND(rp, col, r, threads=threads)
        self.build_s = time.perf_counter() - t0
        self.tau = None
        self.passes = 0

    def step(self):
        """One full SND pass from the current tau (d_s at first); the same
        pass again once converged (Alg. 2 evaluates every r-clique per pass).
        Returns (evaluations, seconds)."""
        t0 = time.perf_counter()
        tau, sweeps, _, ev = self.g.snd(tau=self.tau, max_sweeps=1)
        dt = time.perf_counter() - t0
        self.tau = tau
        self.passes += sweeps
        return ev, dt


def peel_sample(scale: int = PEEL_SAMPLE_SCALE):
    """The single-threaded peeling oracle (Alg. 1) on R-MAT scale `scale`
    (k-truss), the bounded sample of the exact kappa computation."""
    import oracle
    from paper_1704_00386_gb300 import graphs as G
    n, s, d = G.rmat(scale, 16, seed=2)
    rp, col = G.to_csr(n, s, d)
    t0 = time.perf_counter()
    g = oracle.Graph(rp, col, 2, 3, incidence=False)
    g.peel()
    dt = time.perf_counter() - t0
    return {"seconds": dt, "r_cliques": g.num_r, "r_cliques_per_s": g.num_r / dt, "threads": 1,
            "sample": f"R-MAT scale {scale} EF16 k-truss, oracle peeling (Alg. 1, Batagelj-Zaversnik bins)"}


def cpu_baseline(w, rp_h, col_h, threads=0, seconds=CPU_SND_SECONDS):
    """SND passes of the oracle on all host cores on the workload's own graph,
    for about `seconds` (at least one pass), plus the peeling sample."""
    cpu = CpuSND(rp_h, col_h, w["r"], threads)
    ev_tot, dt_tot = 0, 0.0
    while dt_tot < seconds or cpu.passes == 0:
        ev, dt = cpu.step()
        ev_tot += ev
        dt_tot += dt
    peel = peel_sample()
    return {"value": ev_tot / dt_tot, "unit": UNIT, "cores": cpu.g.threads, "kind": "oracle",
            "sample": f"{w['name']} ({w['r']},{w['s']}) itself: {cpu.passes} full SND passes from d_s "
                      f"(oracle arithmetic, loop over r-cliques on {cpu.g.threads} threads); incidence "
                      f"built once beforehand in {cpu.build_s:.1f} s (not timed)",
            "seconds": dt_tot, "evaluations": ev_tot, "incidence_build_s": cpu.build_s,
            "nproc": os.cpu_count(), "peel": peel}


# ------------------------------------------------------------- replicas

def job_rate(local_ms: float, local_units: float, dist=None, device="cpu"):
    """Whole-job throughput of N replicas: the units every rank processed,
    summed, over the slowest rank's time (max over ranks).  Returns (rate per
    second, max ms, total units).  With dist = None, the single-rank values."""
    if dist is None:
        return local_units / (local_ms / 1000.0), float(local_ms), float(local_units)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    ms, units = float(t.item()), float(e.item())
    return units / (ms / 1000.0), ms, units


# ----------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The oracle on the same graph as our arm: each step is one full SND pass
    (Alg. 2) on all host cores; warm-up passes are untimed."""
    if rank != 0:
        return 0
    from paper_1704_00386_gb300 import graphs as G
    w = G.workload(args.workload)
    if not isinstance(w["row_ptr"], np.ndarray):  # generated on a device: bring it to the host
        w = dict(w, row_ptr=w["row_ptr"].cpu().numpy(), col=w["col"].cpu().numpy())
    rp_h, col_h = w["row_ptr"], w["col"]
    cpu = CpuSND(rp_h, col_h, w["r"], args.cpu_threads)
    times, evs = [], []
    for i in range(args.warmup + args.steps):
        ev, dt = cpu.step()
        if i >= args.warmup:
            times.append(dt)
            evs.append(ev)
    value = sum(evs) / sum(times)
    sample = (f"{w['name']} ({w['r']},{w['s']}) itself: one full SND pass per step (oracle arithmetic, "
              f"loop over r-cliques on {cpu.g.threads} threads), continuing from the previous pass; "
              f"incidence built once beforehand in {cpu.build_s:.1f} s (not timed)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(w, rp_h, cpu.g.num_r, cpu.g.num_incidences, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu.g.threads, "kind": "oracle",
                         "sample": sample, "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
    if isinstance(w["row_ptr"], np.ndarray):
        rp_h, col_h = w["row_ptr"], w["col"]
        rp_d = torch.from_numpy(rp_h).to(dev)
        col_d = torch.from_numpy(col_h).to(dev)
    else:  # generated on the device (large R-MAT)
        rp_d, col_d = w["row_ptr"].to(dev), w["col"].to(dev)
        rp_h, col_h = rp_d.cpu().numpy(), col_d.cpu().numpy()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    # r-cliques in no s-clique (d_s = 0): counted as evaluated in every SND pass
    # and in the first AND pass, as in the paper's loops, but never launched
    probe = nd.build_incidence(rp_d, col_d, r, s)
    num_zero = int((probe.s_degree() == 0).sum().item())
    probe.free()
    del probe

    def one_step():
        inc = nd.build_incidence(rp_d, col_d, r, s)
        tau_s, it_s = inc.snd()
        _, ev, ic = inc.last_passes(with_incidences=True)
        ev_s = int(ev.sum())
        snd_bytes = [4.0 * inc.q * float(x) for x in ic]
        snd_rows = [int(x) for x in ev]
        tau_a, it_a, ev_a = inc.and_(notify=True)
        _, ev2, ic2 = inc.last_passes(with_incidences=True)
        info = dict(num_r=inc.num_r, M=inc.num_incidences, q=inc.q, snd_iters=it_s,
                    and_iters=it_a, snd_evals=ev_s, and_evals=ev_a,
                    snd_inc=[int(x) for x in ic], snd_rows=snd_rows,
                    and_inc=[int(x) for x in ic2], and_rows=[int(x) for x in ev2])
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
    value, total_ms_max, evals_all = job_rate(total_ms, evals_rank, dist, dev)

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
    # Algorithmic (compulsory) DRAM bytes of a pass: the incidence ids it
    # streams (4q B each, counted by the kernel) + per evaluated r-clique
    # 24 B (16 B work item, 4 B own tau, 4 B tau write; the first touch of
    # its value as a gathered tau is within the 4 B write) and, for (2,3),
    # 20 B more (8 B CSR positions of the edge, 8 B for its two copies in
    # the gather layout, 4 B first touch of the second copy), for (1,2) 4 B
    # more (the 2 B write of its 16-bit copy and the first touch of it).  The q gathered
    # tau values per incidence are L2 hits while tau fits in L2, so they are
    # not DRAM bytes.
    info = infos[-1]
    peak, peak_kind = load_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, ms) = top
    N_R, M, q = info["num_r"], info["M"], info["q"]
    if name in ("snd_pass", "and_pass"):
        key = "snd" if name == "snd_pass" else "and"
        row_bytes = 44.0 if q == 2 else (28.0 if q == 1 else 24.0)
        tot_bytes = sum(4.0 * q * sum(i[key + "_inc"]) + row_bytes * sum(i[key + "_rows"]) for i in infos)
        eff = sum(len(i[key + "_inc"]) for i in infos)
        per_launch = tot_bytes / max(eff, 1)
        units = (f"4q B x incidences streamed + {row_bytes:.0f} B x r-cliques evaluated, summed over the {eff} "
                 f"effective {key.upper()} passes of the timed steps")
    else:
        eff = launches
        per_launch = 8.0 * M / max(launches, 1) if name == "tri_fill" else float(rp_h[-1]) * 4.0
        units = "8 B per incidence written (fill) or CSR bytes read"
    avg_ms = ms / max(eff, 1)
    achieved = per_launch / (avg_ms / 1000.0) / 1e9
    # DRAM traffic per SND pass: the ncu bytes per incidence of the R-MAT scale 18 k-truss pass,
    # scaled by the incidences of this workload (a full SND pass streams every row); None for any
    # other kernel or once the kernel has changed.
    traffic = None
    if name == "snd_pass" and q == 2 and NCU_SND_TRAFFIC_PER_INCIDENCE is not None:
        traffic = NCU_SND_TRAFFIC_PER_INCIDENCE * M
    # Three byte models of the same pass, each over its measured average time:
    #   frac       compulsory DRAM bytes: 4q B per incidence streamed + the per-row
    #              bytes above (the gathered tau values are L2 hits);
    #   frac_survey every operand counted once, gathers included:
    #              16 B per r-clique + 8q B per incidence (4 B id + 4 B gathered tau);
    #   frac_dram  the DRAM bytes ncu measured (traffic), when known.
    survey_bytes = None
    if name in ("snd_pass", "and_pass"):
        key = "snd" if name == "snd_pass" else "and"
        sb = sum(8.0 * q * sum(i[key + "_inc"]) + 16.0 * sum(i[key + "_rows"]) for i in infos)
        survey_bytes = sb / max(eff, 1)
    survey_gbs = survey_bytes / (avg_ms / 1000.0) / 1e9 if survey_bytes else None
    dram_gbs = traffic / (avg_ms / 1000.0) / 1e9 if traffic else None
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "bytes_per_launch": per_launch, "launches_effective": eff, "avg_launch_ms": avg_ms,
                "units": units,
                "frac_survey": survey_gbs / peak if survey_gbs else None,
                "achieved_survey": survey_gbs,
                "bytes_per_launch_survey": survey_bytes,
                "units_survey": "16 B x r-cliques evaluated + 8q B x incidences streamed (4 B id + 4 B gathered tau)",
                "frac_dram": dram_gbs / peak if dram_gbs else None,
                "achieved_dram": dram_gbs,
                "units_dram": "ncu dram__bytes_read.sum + dram__bytes_write.sum per pass (traffic) / average pass time",
                "note": "gather-bound: the L1 wavefronts of the q tau gathers per incidence set the pace, not DRAM"}

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
        e2e_rate, _, _ = job_rate(1000.0 * dt, ev_total, dist, dev)
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": int(rp_pin.nbytes + col_pin.nbytes),
               "d2h_bytes_per_step": int(out_s.nbytes + out_a.nbytes)}

    # launched evaluations: without the d_s = 0 rows of every SND pass and of the first AND pass
    launched = sum(i["snd_evals"] - num_zero * len(i["snd_rows"]) + i["and_evals"] - num_zero * (1 if i["and_rows"] else 0)
                   for i in infos)
    value_launched, _, _ = job_rate(total_ms, launched, dist, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, rp_h, col_h, args.cpu_threads)

    extra = None
    if rank == 0 and world == 1 and not args.no_extras:
        extra = run_extras(args, dev)

    if rank == 0:
        phases = {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": workload_config(w, rp_h, N_R, M, world),
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "gpu_launches": int(sum(v[0] for v in prof.values())),
            "clocks": clk,
            "per_step": {"snd_iters": info["snd_iters"], "and_iters": info["and_iters"],
                         "snd_evals": info["snd_evals"], "and_evals": info["and_evals"],
                         "and_incidences": sum(info["and_inc"]), "snd_incidences": sum(info["snd_inc"]),
                         "zero_ds_r_cliques": num_zero,
                         "launched_evals": (info["snd_evals"] - num_zero * len(info["snd_rows"]) +
                                            info["and_evals"] - num_zero * (1 if info["and_rows"] else 0)),
                         "step_ms": step_ms},
            "value_launched": value_launched,
            "value_launched_note": "h-index evaluations actually launched (d_s = 0 rows excluded) / device time",
            "extra": extra,
            "kernels": phases,
            "parity_vs_oracle_digest": parity, "snd_equals_and": same,
        }
        print(json.dumps(line), flush=True)
    return 0


def _evals_of(inc, and_evals):
    _, ev = inc.last_passes()
    return int(ev.sum()) + int(and_evals)


def run_batch(args):
    """The batched workload, the whole list (default 4,096 graphs): one
    disjoint-union batch against one graph per launch, same GPU."""
    import torch
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    print(json.dumps(batch_measure(args.batch_count, steps=args.steps, autotune=True)), flush=True)
    return 0


SERVE_BUDGET = 64 << 30


def serve_requests(count: int, seed: int = 5):
    """The served workload: graphs with 1K-2M edges (log-uniform), family uniform
    over ER / Chung-Lu / R-MAT, job uniform over (1,2) / (2,3) / (3,4) ((3,4)
    only where the footprint bound fits an eighth of the budget, else (2,3))."""
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import serve
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = np.exp(rng.uniform(np.log(1e3), np.log(2e6), size=count))
    reqs = []
    for i, e in enumerate(edges):
        fam = int(rng.integers(0, 3))
        n = max(16, int(e * 2 / 8))
        sd = 5_000_000 + i
        if fam == 0:
            a, b = G.erdos_renyi(n, 8.0 / (n - 1), seed=sd)
        elif fam == 1:
            a, b = G.chung_lu(n, 2.2, 8.0, seed=sd)
        else:
            _, a, b = G.rmat(max(1, int(np.ceil(np.log2(n)))), 8, seed=sd, n_limit=n)
        rp, col = G.to_csr(n, a, b)
        r, s_ = [(1, 2), (2, 3), (3, 4)][int(rng.integers(0, 3))]
        if (r, s_) == (3, 4) and serve.footprint_bytes(rp, col, 3) > SERVE_BUDGET // 8:
            r, s_ = 2, 3
        reqs.append((rp, col, r, s_))
    return reqs


def serve_measure(reqs, loads=(0.5, 0.7, 0.9)):
    """Saturated throughput, then p50/p99 latency at each load (a fraction of
    saturation), against one-request-at-a-time service; every result checked
    against the result served alone."""
    from paper_1704_00386_gb300 import serve

    def run_stream(arrivals, workers, batching=True):
        srv = serve.Server(budget_bytes=SERVE_BUDGET, workers=workers, batch_bytes=(1 << 30) if batching else 1,
                           max_batch=64 if batching else 1)
        hs = []
        t0 = time.perf_counter()
        for (rp, col, r, s_), at in zip(reqs, arrivals):
            d = t0 + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            hs.append(srv.submit(rp, col, r, s_, "and"))
        srv.close()
        span = max(h.finish for h in hs) - t0
        return hs, span

    zero = np.zeros(len(reqs))
    run_stream(zero[:8], 4)                               # warm-up
    hs, span = run_stream(zero, 4)
    sat = len(reqs) / span
    base_hs, base_span = run_stream(zero, 1, batching=False)
    alone = {i: h.result for i, h in enumerate(base_hs)}
    same = all(np.array_equal(h.result, alone[i]) for i, h in enumerate(hs))
    out = {"metric": METRIC, "mode": "serve", "requests": len(reqs),
           "edges_total": int(sum(int(rp[-1]) // 2 for rp, _, _, _ in reqs)),
           "saturated_requests_per_s": sat, "one_at_a_time_requests_per_s": len(reqs) / base_span,
           "saturated_latency": serve.latency_stats(hs), "results_identical_to_one_at_a_time": bool(same),
           "load": {}}
    for frac in loads:
        arr = serve.poisson_arrivals(frac * sat, len(reqs), seed=int(frac * 100))
        hs2, span2 = run_stream(arr, 4)
        same2 = all(np.array_equal(h.result, alone[i]) for i, h in enumerate(hs2))
        out["load"][str(frac)] = {"rate_per_s": frac * sat, "throughput_per_s": len(reqs) / span2,
                                  "latency": serve.latency_stats(hs2), "results_identical": bool(same2),
                                  "batched_requests": int(sum(h.batched_with > 1 for h in hs2))}
    return out


def run_serve(args):
    """The served workload: a Poisson stream of graphs with 1K-2M edges, mixed
    jobs; saturated throughput, then p50/p99 latency at 0.5 / 0.7 / 0.9 of
    it; one-request-at-a-time service as the baseline."""
    import torch
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    print(json.dumps(serve_measure(serve_requests(args.requests))), flush=True)
    return 0


def batch_measure(count: int, steps: int = 1, autotune: bool = False):
    """The batched workload: `count` independent graphs (ER / Chung-Lu / R-MAT, n
    in [100, 50000]), core and truss numbers for each: one disjoint-union
    batch against one graph per launch, same GPU, results compared.  With
    autotune, the batch handle's buckets are tuned (nd_autotune) first; the
    tuned thresholds are cached for the size class and every later build of
    the batch starts with them."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    workers = max(1, min(16, os.cpu_count() or 1))
    t0 = time.perf_counter()
    gs = G.batch_graphs(count, seed=4, workers=workers)
    gen_s = time.perf_counter() - t0
    dev = [(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()) for rp, col, _ in gs]
    stream = torch.cuda.current_stream()
    out = {"metric": METRIC, "unit": UNIT, "mode": "batch", "graphs": len(gs),
           "edges": int(sum(int(rp[-1]) // 2 for rp, _, _ in gs)), "generation_s": gen_s,
           "autotuned": bool(autotune), "jobs": {}}

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        return res, e0.elapsed_time(e1)

    for r, s in ((1, 2), (2, 3)):
        def plain():
            ev, taus = 0, []
            for rp, col in dev:
                inc = nd.build_incidence(rp, col, r, s)
                t, _ = inc.snd()
                ev_s = _evals_of(inc, 0)
                ta, _, ev_a = inc.and_(notify=True)
                ev += ev_s + ev_a
                taus.append(t)
                inc.free()
            return ev, taus

        def batched():
            inc, offs = nd.build_incidence_batch(dev, r, s)
            t, _ = inc.snd()
            ev_s = _evals_of(inc, 0)
            ta, _, ev_a = inc.and_(notify=True)
            inc.free()
            return ev_s + ev_a, (t, offs)

        thr = None
        if autotune:
            inc, _ = nd.build_incidence_batch(dev, r, s)
            thr, _ = inc.autotune(passes=2)
            inc.free()
        batched()                                 # warm-up
        nd.prof_enable(True)
        (ev_b, (tb, offs)), ms_b = timed(batched)
        prof = nd.prof_read()
        nd.prof_enable(False)
        ms_bs = [ms_b]
        for _ in range(max(0, steps - 1)):
            _, ms = timed(batched)
            ms_bs.append(ms)
        plain()                                   # warm-up
        (ev_p, taus), ms_p = timed(plain)
        same = all(torch.equal(taus[i], tb[offs[i]:offs[i + 1]]) for i in range(len(dev)))
        ms_b = statistics.median(ms_bs)
        out["jobs"][f"({r},{s})"] = {
            "batched_ms": ms_b, "batched_updates_per_s": ev_b / (ms_b / 1e3),
            "batched_graphs_per_s": len(dev) / (ms_b / 1e3),
            "plain_ms": ms_p, "plain_updates_per_s": ev_p / (ms_p / 1e3),
            "plain_graphs_per_s": len(dev) / (ms_p / 1e3),
            "speedup": ms_p / ms_b, "results_identical": bool(same),
            "thresholds": list(thr) if thr else None,
            "batched_kernels_ms": {k: round(v[1], 2) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]}}
    return out


def core26_measure(steps: int = 1):
    """The k-core of R-MAT scale 26, EF 16 (67M vertices, 2.1G CSR
    entries), generated on the device: build + SND + AND per step."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    t0 = time.perf_counter()
    w = G.workload("rmat_core_s26_ef16")
    rp, col = w["row_ptr"].cuda(), w["col"].cuda()
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def one():
        inc = nd.build_incidence(rp, col, 1, 2)
        t_s, it_s = inc.snd()
        _, ev = inc.last_passes()
        t_a, it_a, ev_a = inc.and_(notify=True)
        inc.free()
        return int(ev.sum()) + ev_a, it_s, it_a, t_s, t_a

    one()                                         # warm-up
    ms, res = [], None
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = one()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ev, it_s, it_a, t_s, t_a = res
    out = {"workload": w["name"], "recipe": w["recipe"], "n": int(rp.numel() - 1), "nnz": int(col.numel()),
           "generation_s": gen_s, "ms_per_step": statistics.median(ms), "steps": steps,
           "updates_per_s": ev / (statistics.median(ms) / 1e3), "snd_iters": it_s, "and_iters": it_a,
           "snd_equals_and": bool(torch.equal(t_s, t_a))}
    del rp, col, w
    torch.cuda.empty_cache()
    return out


def run_extras(args, dev):
    """After the timed region: SND / AND / AND-nn on the three single-graph
    workloads, one scale-26 k-core step, a 256-graph batch (autotuned)
    against one graph per launch, and a 64-request stream at half of its
    saturated rate.  Each is
    reported, none changes the headline."""
    import torch
    extra = {}
    for key, fn in (("sweeps", lambda: sweeps_measure(reps=1)),
                    ("rmat_core_s26_ef16", lambda: core26_measure(1)),
                    ("batch_256", lambda: batch_measure(256, steps=1, autotune=True)),
                    ("serve_64", lambda: serve_measure(serve_requests(64), loads=(0.5,)))):
        t0 = time.perf_counter()
        try:
            extra[key] = fn()
        except Exception as e:  # reported, never fatal to the headline
            extra[key] = {"error": f"{type(e).__name__}: {e}"}
        extra[key]["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize(dev)
    return extra


SWEEP_WORKLOADS = ("chunglu_n2000_g2.5_d10", "rmat_s20_ef16", "chunglu_n100000_g2.1_d20_planted200")


def sweeps_measure(names=SWEEP_WORKLOADS, reps=3):
    """SND, AND with notification and AND without it (the paper's AND-nn),
    each from d_s to convergence on one built incidence: updating passes,
    evaluations and device time (median of reps), and AND-nn / AND time, the
    ratio the paper tabulates for its CPU runs."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        return res, e0.elapsed_time(e1)

    out = {}
    for name in names:
        w = G.workload(name)
        rp = torch.from_numpy(np.asarray(w["row_ptr"])).cuda()
        col = torch.from_numpy(np.asarray(w["col"])).cuda()
        inc = nd.build_incidence(rp, col, w["r"], w["s"])
        rec = {"r": w["r"], "s": w["s"], "r_cliques": inc.num_r}
        kappa = None
        for mode in ("snd", "and", "and_nn"):
            runs = []
            for _ in range(reps):
                if mode == "snd":
                    (tau, it), ms = timed(inc.snd)
                    ev = _evals_of(inc, 0)
                else:
                    (tau, it, ev), ms = timed(lambda: inc.and_(notify=(mode == "and")))
                runs.append((ms, it, ev))
                if kappa is None:
                    kappa = tau.clone()
                elif not torch.equal(tau, kappa):
                    rec["error"] = f"{mode} differs from SND"
            ms = statistics.median(r[0] for r in runs)
            rec[mode] = {"passes": runs[-1][1], "evaluations": runs[-1][2], "ms": ms,
                         "updates_per_s": runs[-1][2] / (ms / 1e3) if ms > 0 else None}
        rec["and_nn_over_and_time"] = rec["and_nn"]["ms"] / rec["and"]["ms"] if rec["and"]["ms"] > 0 else None
        inc.free()
        out[name] = rec
    return out


def run_sweeps(args):
    import torch
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    names = SWEEP_WORKLOADS if args.workload == "rmat_s20_ef16" else (args.workload,)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "mode": "sweeps", "workloads": sweeps_measure(names)}),
          flush=True)
    return 0


def run_otf(args):
    """The stored incidence against the no-storage mode (ND_BUILD_ON_THE_FLY)
    on one workload: build, SND and AND times, memory held by the handle."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    w = G.workload(args.workload)
    rp = torch.from_numpy(w["row_ptr"]).cuda()
    col = torch.from_numpy(w["col"]).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        return res, e0.elapsed_time(e1)

    out = {"metric": METRIC, "unit": UNIT, "mode": "otf", "workload": args.workload, "r": w["r"], "s": w["s"]}
    kappa = {}
    for name, otf in (("stored", False), ("on_the_fly", True)):
        inc = nd.build_incidence(rp, col, w["r"], w["s"], on_the_fly=otf)  # warm-up
        inc.snd()
        inc.free()
        inc, ms_build = timed(lambda: nd.build_incidence(rp, col, w["r"], w["s"], on_the_fly=otf))
        (tau, iters), ms_snd = timed(inc.snd)
        ev_s = _evals_of(inc, 0)
        (ta, it_a, ev_a), ms_and = timed(lambda: inc.and_(notify=True))
        kappa[name] = tau
        out[name] = {"build_ms": ms_build, "snd_ms": ms_snd, "snd_ms_per_pass": ms_snd / (iters + 1),
                     "and_ms": ms_and, "updates_per_s": (ev_s + ev_a) / ((ms_snd + ms_and) / 1e3),
                     "handle_bytes": inc.incidence_bytes(), "snd_equals_and": bool(torch.equal(tau, ta))}
        inc.free()
    out["results_identical"] = bool(torch.equal(kappa["stored"], kappa["on_the_fly"]))
    print(json.dumps(out), flush=True)
    return 0


def run_quality(args):
    """Section 5.2: how close the early-stopped iterates are to kappa, per
    pass, as Kendall's tau-b against kappa and as the fraction of r-cliques
    already at kappa (SND, and AND with notification)."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    w = G.workload(args.workload)
    rp = torch.from_numpy(w["row_ptr"]).cuda()
    col = torch.from_numpy(w["col"]).cuda()
    inc = nd.build_incidence(rp, col, w["r"], w["s"])
    kappa, iters = inc.snd()
    out = {"mode": "quality", "workload": args.workload, "r": w["r"], "s": w["s"], "snd_iters": iters,
           "kendall_tau_b": {}, "accuracy": {}}
    for mode in ("snd", "and"):
        kt, acc = [], []
        for k in range(0, iters + 1):
            tk, _ = inc.iterate_k(mode, k)
            kt.append(nd.kendall_tau_b(tk, kappa))
            acc.append(nd.count_equal(tk, kappa) / max(inc.num_r, 1))
        out["kendall_tau_b"][mode] = kt
        out["accuracy"][mode] = acc
        out[f"{mode}_passes_to_kendall_0.90"] = next((k for k, v in enumerate(kt) if v >= 0.9), None)
    print(json.dumps(out), flush=True)
    return 0


def run_noalloc(args):
    """The allocation-free k-core entry point (nd_core_snd_noalloc) against
    nd_build_incidence(1,2) + nd_snd on the largest graph it accepts, R-MAT
    scale 20 EF16 (1,048,576 vertices): time per run and per pass."""
    import torch
    from paper_1704_00386_gb300 import graphs as G
    from paper_1704_00386_gb300 import nd
    torch.cuda.set_device(0)
    nd.load(build_if_missing=False)
    n, s, d = G.rmat(20, 16, seed=2)
    rp, col = G.to_csr(n, s, d)
    rp_d, col_d = torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn, reps=3):
        best, res = None, None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return res, best

    nd.core_snd_noalloc(rp_d[:1], col_d[:0])  # the set-up call (n = 0)
    (core_a, it_a), ms_a = timed(lambda: nd.core_snd_noalloc(rp_d, col_d))

    def alloc_path():
        inc = nd.build_incidence(rp_d, col_d, 1, 2)
        t, it = inc.snd()
        inc.free()
        return t, it

    (core_b, it_b), ms_b = timed(alloc_path)
    inc = nd.build_incidence(rp_d, col_d, 1, 2)
    _, ms_snd = timed(lambda: inc.snd())
    inc.free()
    print(json.dumps({"mode": "noalloc", "n": n, "nnz": int(rp[-1]), "max_degree": int(np.diff(rp).max()),
                      "passes": it_a, "noalloc_ms": ms_a, "build_plus_snd_ms": ms_b, "snd_only_ms": ms_snd,
                      "noalloc_ms_per_pass": ms_a / (it_a + 1), "snd_ms_per_pass": ms_snd / (it_b + 1),
                      "results_identical": bool(torch.equal(core_a, core_b)) and it_a == it_b}), flush=True)
    return 0


def main():
    args = parse()
    if args.mode == "sweeps":
        return run_sweeps(args)
    if args.mode == "noalloc":
        return run_noalloc(args)
    if args.mode == "otf":
        return run_otf(args)
    if args.mode == "quality":
        return run_quality(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
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

"""Write tests/golden/digests.json: expected results at full workload sizes.

Calls only the CPU oracle (``oracle/``) and the seeded generators.  For each
named workload it records SHA-256 digests of the input CSR, of the canonical
r-clique tuples, of d_s (= tau_0), of kappa_s (peeling, Alg. 1), and of the
SND iterates tau_1 and tau_2 (Alg. 2), plus a few summary numbers.  The GPU
parity tests recompute the same digests from the CUDA path and compare them,
which is a bit-exact comparison of every element.

Usage: python tests/golden/make_digests.py [workload ...]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1704_00386_gb300 import graphs as G  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "digests.json")
WORKLOADS = ["chunglu_n2000_g2.5_d10", "chunglu_n100000_g2.1_d20_planted200", "rmat_s20_ef16"]


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<")).tobytes()).hexdigest()


def csr_digest(rp, col) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rp, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(col, dtype="<i4").tobytes())
    return h.hexdigest()


def sample_idx(num: int, k: int = 64) -> list:
    rng = np.random.Generator(np.random.PCG64(12345))
    if num == 0:
        return []
    return sorted(set(rng.integers(0, num, size=k).tolist()))


def one(name: str) -> dict:
    t0 = time.time()
    w = G.workload(name)
    rp, col, r, s = w["row_ptr"], w["col"], w["r"], w["s"]
    rec = {"recipe": w["recipe"], "r": r, "s": s, "n": int(rp.size - 1), "nnz": int(rp[-1]),
           "csr_sha256": csr_digest(rp, col)}
    g = oracle.Graph(rp, col, r, s, incidence=False)
    rec["num_r"] = g.num_r
    rec["r_cliques_sha256"] = sha(g.r_cliques())
    ds = g.s_degree()
    rec["num_incidences"] = int(ds.astype(np.int64).sum())
    rec["ds_sha256"] = sha(ds)
    rec["ds_max"] = int(ds.max()) if ds.size else 0
    kap = g.peel()
    rec["kappa_sha256"] = sha(kap)
    rec["kappa_max"] = int(kap.max()) if kap.size else 0
    rec["kappa_sum"] = int(kap.astype(np.int64).sum())
    idx = sample_idx(g.num_r)
    rec["sample_idx"] = idx
    rec["kappa_sample"] = [int(kap[i]) for i in idx]
    del g
    gi = oracle.Graph(rp, col, r, s, incidence=True)
    for k in (1, 2):
        tk = gi.snd(max_sweeps=k)[0]
        rec[f"snd_tau{k}_sha256"] = sha(tk)
    if gi.num_r <= 200000:
        _, sweeps, updating, evals = gi.snd()
        rec["snd_updating_sweeps"] = updating
    rec["oracle_seconds"] = round(time.time() - t0, 1)
    return rec


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["_about"] = ("Written by tests/golden/make_digests.py from the CPU oracle only "
                      "(peeling, Alg. 1; SND, Alg. 2). Digests are SHA-256 of little-endian "
                      "int32 arrays (int64 row_ptr + int32 col for the CSR).")
    for name in names:
        rec = one(name)
        data[name] = rec
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(name, rec["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or WORKLOADS)

"""Seeded synthetic graph generators and CSR normalisation.

This module holds no part of the decomposition method: it only draws graphs
and writes them as simple, symmetric, sorted CSR (row_ptr int64[n+1],
col int32[2m]).  Both the CPU oracle tests and the CUDA path read graphs made
here, so the two sides always see the same input.

The paper measures on SNAP / Network Repository graphs (Section 5, Table 2).
Those are replaced by synthetic graphs with the same character: power-law
social graphs (Chung-Lu), skewed web-like graphs (R-MAT), Erdos-Renyi graphs,
and planted cliques that create deep (3,4)-nuclei.

Generator readings (the workloads leave these open):
* Chung-Lu: weight w_i = (i + 1) ** (-1 / (gamma - 1)), scaled so that
  sum(w) = n * mean_degree, each weight capped at sqrt(sum(w)); n*d/2
  endpoint pairs are drawn independently with probability proportional to w;
  self-loops and duplicates are dropped; vertex labels are then randomly
  permuted so that ids carry no degree information.
* R-MAT: the Graph500 recursive quadrant choice with (a, b, c, d) and no
  noise; EF * 2**scale directed samples; symmetrised, deduplicated, loops
  dropped, labels randomly permuted.
* Erdos-Renyi: G(n, p) drawn exactly by sampling Binomial(n(n-1)/2, p)
  distinct pairs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "to_csr", "chung_lu", "rmat", "erdos_renyi", "plant_cliques",
    "graph_from_edges", "toy_core_graph", "complete_graph", "cycle_graph",
    "star_graph", "disjoint_union", "hub_graph", "batch_graphs", "workload",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_csr(n: int, src, dst):
    """Simple undirected CSR from an arbitrary directed pair list.

    Drops self-loops, symmetrises, removes duplicates and sorts each row.
    Returns (row_ptr int64[n+1], col int32[nnz]).
    """
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    if src.size:
        if src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n:
            raise ValueError("vertex id out of range")
    keep = src != dst
    src, dst = src[keep], dst[keep]
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    up = _sorted_unique(lo * np.int64(n) + hi)      # (lo, hi) pairs, sorted by lo then hi
    dn = np.sort((up % n) * np.int64(n) + up // n)  # (hi, lo) pairs, sorted by hi then lo
    up_u, up_v = up // n, up % n
    dn_u, dn_v = dn // n, dn % n
    cnt_up = np.bincount(up_u, minlength=n).astype(np.int64)
    cnt_dn = np.bincount(dn_u, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(cnt_up + cnt_dn)
    # a row is its smaller neighbours (all < u) followed by its larger ones (all > u)
    start_up = np.zeros(n, np.int64)
    start_up[1:] = np.cumsum(cnt_up)[:-1]
    start_dn = np.zeros(n, np.int64)
    start_dn[1:] = np.cumsum(cnt_dn)[:-1]
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    i_dn = np.arange(dn.size, dtype=np.int64)
    col[row_ptr[dn_u] + (i_dn - start_dn[dn_u])] = dn_v
    i_up = np.arange(up.size, dtype=np.int64)
    col[row_ptr[up_u] + cnt_dn[up_u] + (i_up - start_up[up_u])] = up_v
    return row_ptr, col


def _sorted_unique(a):
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _relabel(n: int, rng: np.random.Generator, src, dst):
    perm = rng.permutation(n).astype(np.int64)
    return perm[src], perm[dst]


def chung_lu(n: int, gamma: float, mean_degree: float, seed: int):
    """Chung-Lu power-law graph (expected degrees follow exponent gamma)."""
    rng = _rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    w *= n * mean_degree / w.sum()
    cap = np.sqrt(w.sum())
    w = np.minimum(w, cap)
    p = w / w.sum()
    m = int(round(n * mean_degree / 2.0))
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    src = np.searchsorted(cdf, rng.random(m), side="right")
    dst = np.searchsorted(cdf, rng.random(m), side="right")
    src = np.minimum(src, n - 1)
    dst = np.minimum(dst, n - 1)
    src, dst = _relabel(n, rng, src, dst)
    return src, dst


def rmat(scale: int, edge_factor: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0,
         n_limit: int | None = None):
    """R-MAT directed samples (Graph500 quadrant recursion, no noise).

    Returns (n, src, dst).  With ``n_limit`` the vertex set is cut to the
    first n_limit ids before relabelling and samples touching larger ids are
    rejected (used for graph sizes that are not a power of two).
    """
    a, b, c, d = abcd
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    rng = _rng(seed)
    ne = edge_factor * (1 << scale)
    src = np.zeros(ne, dtype=np.int64)
    dst = np.zeros(ne, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    chunk = 1 << 22
    for lo in range(0, ne, chunk):
        hi = min(ne, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.int64)
        t = np.zeros(hi - lo, dtype=np.int64)
        for level in range(scale):
            r = rng.random(hi - lo)
            sbit = r >= ab
            tbit = ((r >= a) & (r < ab)) | (r >= abc)
            s |= sbit.astype(np.int64) << level
            t |= tbit.astype(np.int64) << level
        src[lo:hi] = s
        dst[lo:hi] = t
    n = 1 << scale
    if n_limit is not None and n_limit < n:
        keep = (src < n_limit) & (dst < n_limit)
        src, dst = src[keep], dst[keep]
        n = n_limit
    src, dst = _relabel(n, rng, src, dst)
    return n, src, dst


def erdos_renyi(n: int, p: float, seed: int):
    """G(n, p): each of the n(n-1)/2 pairs present independently with p."""
    rng = _rng(seed)
    total = n * (n - 1) // 2
    m = int(rng.binomial(total, p)) if total else 0
    picked = _sorted_unique(rng.integers(0, total, size=int(m * 1.1) + 16, dtype=np.int64))
    while picked.size < m:
        more = rng.integers(0, total, size=m - picked.size + 16, dtype=np.int64)
        picked = _sorted_unique(np.concatenate([picked, more]))
    picked = rng.permutation(picked)[:m]
    # unrank pair index k -> (i, j), i < j, rows of length n-1-i
    k = picked.astype(np.float64)
    i = np.floor((2 * n - 1 - np.sqrt((2 * n - 1) ** 2 - 8 * k)) / 2).astype(np.int64)
    row_start = i * (2 * n - i - 1) // 2
    over = picked < row_start
    i[over] -= 1
    row_start = i * (2 * n - i - 1) // 2
    under = picked >= row_start + (n - 1 - i)
    i[under] += 1
    row_start = i * (2 * n - i - 1) // 2
    j = picked - row_start + i + 1
    return i, j


def plant_cliques(n: int, count: int, size_lo: int, size_hi: int, seed: int):
    """Edges of `count` cliques, sizes uniform in [size_lo, size_hi], each on
    a uniformly random vertex set."""
    rng = _rng(seed)
    src, dst = [], []
    for _ in range(count):
        k = int(rng.integers(size_lo, size_hi + 1))
        vs = rng.choice(n, size=k, replace=False).astype(np.int64)
        a, b = np.triu_indices(k, 1)
        src.append(vs[a])
        dst.append(vs[b])
    if not src:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(src), np.concatenate(dst)


def hub_graph(n: int = 3000, hubs: int = 6, seed: int = 107):
    """Sparse Erdos-Renyi background (mean degree 6), `hubs` mutually adjacent
    hub vertices each joined to 70-85% of the others, and 5 planted cliques
    of size 20-40: long incidence rows for every (r,s) (hub degrees, hub-hub
    edge triangles and hub-triple 4-cliques all exceed 1024)."""
    rng = _rng(seed)
    i, j = erdos_renyi(n, 6.0 / (n - 1), seed=seed)
    src, dst = [i], [j]
    for h in range(hubs):
        k = int(rng.integers(int(0.7 * n), int(0.85 * n)))
        nb = rng.choice(np.arange(hubs, n), size=k, replace=False)
        src.append(np.full(k, h, dtype=np.int64))
        dst.append(nb.astype(np.int64))
    a, b = np.triu_indices(hubs, 1)
    src.append(a)
    dst.append(b)
    s2, d2 = plant_cliques(n, 5, 20, 40, seed=seed + 1)
    src.append(s2)
    dst.append(d2)
    return to_csr(n, np.concatenate(src), np.concatenate(dst))


def _batch_one(args):
    i, n, fam, seed = args
    sd = seed * 1_000_003 + i
    if fam == 0:
        a, b = erdos_renyi(n, 8.0 / (n - 1), seed=sd)
        name = "er"
    elif fam == 1:
        a, b = chung_lu(n, 2.2, 8.0, seed=sd)
        name = "chunglu"
    else:
        scale = max(1, int(np.ceil(np.log2(n))))
        _, a, b = rmat(scale, 8, seed=sd, n_limit=n)
        name = "rmat"
    rp, col = to_csr(n, a, b)
    return rp, col, name


def batch_graphs(count: int, seed: int = 4, n_lo: int = 100, n_hi: int = 50000, workers: int = 1):
    """Independent graphs for batched runs: n uniform in [n_lo, n_hi]; each
    graph is, with probability 1/3 each, Erdos-Renyi with mean degree 8,
    Chung-Lu with exponent 2.2 and mean degree 8, or R-MAT with edge factor 8
    at scale ceil(log2 n) keeping only endpoints below n.  Graph i uses seed
    seed*1_000_003 + i, so the list does not depend on `workers` (processes
    started with spawn).  Returns a list of (row_ptr, col, family)."""
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    fam = rng.integers(0, 3, size=count)
    jobs = [(i, int(ns[i]), int(fam[i]), seed) for i in range(count)]
    if workers <= 1 or count < 2 * workers:
        return [_batch_one(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_one, jobs, chunksize=max(1, count // (8 * workers))))


# ---------------------------------------------------------------------------
# Large R-MAT graphs, generated with torch on any device.  The random numbers
# come from a counter-based hash (SplitMix64's finaliser applied to
# seed * 2**40 + sample * 64 + level), so the same graph comes out on the CPU
# and on a GPU.  Quadrants are chosen by integer comparison of the hash's top
# 53 bits with floor(p * 2**53); vertex labels are scrambled by the bijection
# v -> (v * 0x9E3779B97F4A7C15 + seed) mod 2**scale (odd multiplier).
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def _to_i64(x: int) -> int:
    x &= _M64
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl(t, k: int):
    """Logical right shift of an int64 tensor holding 64-bit patterns."""
    import torch
    return (t >> k) & torch.tensor(_to_i64((1 << (64 - k)) - 1), dtype=torch.int64, device=t.device)


def _splitmix(t):
    import torch
    c1 = torch.tensor(_to_i64(0xBF58476D1CE4E5B9), dtype=torch.int64, device=t.device)
    c2 = torch.tensor(_to_i64(0x94D049BB133111EB), dtype=torch.int64, device=t.device)
    t = t ^ _srl(t, 30)
    t = t * c1
    t = t ^ _srl(t, 27)
    t = t * c2
    return t ^ _srl(t, 31)


def rmat_torch(scale: int, edge_factor: int, seed: int, abcd=(0.57, 0.19, 0.19, 0.05), device="cpu",
               chunk: int = 1 << 26):
    """R-MAT samples as torch int64 (src, dst) on `device`; see the notes above."""
    import torch
    a, b, c, _ = abcd
    th_a = int(a * (1 << 53))
    th_ab = int((a + b) * (1 << 53))
    th_abc = int((a + b + c) * (1 << 53))
    ne = edge_factor * (1 << scale)
    n = 1 << scale
    src = torch.empty(ne, dtype=torch.int64, device=device)
    dst = torch.empty(ne, dtype=torch.int64, device=device)
    mult = torch.tensor(_to_i64(0x9E3779B97F4A7C15), dtype=torch.int64, device=device)
    for lo in range(0, ne, chunk):
        hi = min(ne, lo + chunk)
        idx = torch.arange(lo, hi, dtype=torch.int64, device=device)
        s_ = torch.zeros(hi - lo, dtype=torch.int64, device=device)
        d_ = torch.zeros(hi - lo, dtype=torch.int64, device=device)
        for level in range(scale):
            key = idx * 64 + level + seed * (1 << 40)
            r = _srl(_splitmix(key), 11)  # 53 bits
            sbit = (r >= th_ab).to(torch.int64)
            tbit = (((r >= th_a) & (r < th_ab)) | (r >= th_abc)).to(torch.int64)
            s_ |= sbit << level
            d_ |= tbit << level
        src[lo:hi] = (s_ * mult + seed) & (n - 1)
        dst[lo:hi] = (d_ * mult + seed) & (n - 1)
    return n, src, dst


def to_csr_torch(n: int, src, dst):
    """to_csr on torch tensors (any device): simple, symmetric, sorted CSR
    as (row_ptr int64[n+1], col int32[nnz]) on the same device."""
    import torch
    keep = src != dst
    lo = torch.minimum(src[keep], dst[keep])
    hi = torch.maximum(src[keep], dst[keep])
    del keep
    key = torch.unique(lo * n + hi)  # sorted
    del lo, hi
    u = torch.cat([key // n, key % n])
    v = torch.cat([key % n, key // n])
    del key
    key2, _ = torch.sort(u * n + v)
    del u, v
    row = key2 // n
    col = (key2 % n).to(torch.int32)
    del key2
    counts = torch.bincount(row, minlength=n)
    del row
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=col.device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr, col


def graph_from_edges(n: int, edges):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return to_csr(n, e[:, 0], e[:, 1])


def toy_core_graph():
    """The six-vertex k-core example traced in Section 4 (Figures 5 and 6).

    Vertices a..f are 0..5; edges a-b, a-e, b-c, b-d, c-d, e-f.  The edge set
    follows from the traces: b's neighbours are a, c, d; a's are e and b;
    e notifies a and f.
    """
    a, b, c, d, e, f = range(6)
    return graph_from_edges(6, [(a, b), (a, e), (b, c), (b, d), (c, d), (e, f)])


def complete_graph(k: int):
    a, b = np.triu_indices(k, 1)
    return to_csr(k, a, b)


def cycle_graph(k: int):
    a = np.arange(k)
    return to_csr(k, a, (a + 1) % k)


def star_graph(leaves: int):
    return to_csr(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1))


def disjoint_union(*graphs):
    rps, cols, off = [np.zeros(1, np.int64)], [], 0
    base = 0
    for rp, col in graphs:
        rps.append(rp[1:] + base)
        cols.append(col.astype(np.int64) + off)
        base += int(rp[-1])
        off += rp.size - 1
    return np.concatenate(rps).astype(np.int64), np.concatenate(cols).astype(np.int32)


def number_by_degree_class(row_ptr, col):
    """The same graph with its vertices renumbered by degree class: classes
    floor(log2(degree)) in descending order, isolated vertices last, the old
    order kept inside a class.  Returns (row_ptr, col, new_id_of_old)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col)
    n = row_ptr.size - 1
    deg = np.diff(row_ptr)
    cls = np.where(deg > 0, np.floor(np.log2(np.maximum(deg, 1))).astype(np.int64) + 1, 0)
    order = np.lexsort((np.arange(n), -cls))       # old ids, in their new order
    new_of_old = np.empty(n, dtype=np.int64)
    new_of_old[order] = np.arange(n)
    src = np.repeat(np.arange(n), deg)
    rp, c = to_csr(n, new_of_old[src], new_of_old[col.astype(np.int64)])
    return rp, c, new_of_old


def workload(name: str):
    """Named synthetic workloads, each with its (r, s) job.

    Returns dict(name, r, s, row_ptr, col, recipe).
    """
    if name == "chunglu_n2000_g2.5_d10":
        src, dst = chung_lu(2000, 2.5, 10.0, seed=1)
        rp, col = to_csr(2000, src, dst)
        return dict(name=name, r=1, s=2, row_ptr=rp, col=col,
                    recipe="Chung-Lu n=2000 gamma=2.5 mean degree 10 seed 1; k-core (1,2)")
    if name.startswith("rmat_s") and "_ef" in name:
        # rmat_s{scale}_ef{ef}, e.g. rmat_s20_ef16
        scale = int(name.split("_s")[1].split("_")[0])
        ef = int(name.split("_ef")[1].split("_")[0])
        n, src, dst = rmat(scale, ef, seed=2)
        rp, col = to_csr(n, src, dst)
        recipe = (f"R-MAT scale {scale} edge factor {ef} (0.57,0.19,0.19,0.05) seed 2, "
                  "symmetrised, deduplicated, no loops; k-truss (2,3)")
        if name.endswith("_byclass"):
            # rmat_s{scale}_ef{ef}_byclass: the same graph, vertices numbered by degree class
            rp, col, _ = number_by_degree_class(rp, col)
            recipe += "; vertices renumbered by descending log2-degree class (stable)"
        return dict(name=name, r=2, s=3, row_ptr=rp, col=col, recipe=recipe)
    if name.startswith("rmat_core_s") and "_ef" in name:
        # rmat_core_s{scale}_ef{ef}: k-core of a large R-MAT graph, generated with torch
        # (on the GPU when one is present, else on the CPU); arrays stay torch tensors
        import torch
        scale = int(name.split("_s")[1].split("_")[0])
        ef = int(name.split("_ef")[1].split("_")[0])
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        n, src, dst = rmat_torch(scale, ef, seed=5, device=dev)
        rp, col = to_csr_torch(n, src, dst)
        return dict(name=name, r=1, s=2, row_ptr=rp, col=col,
                    recipe=f"R-MAT scale {scale} edge factor {ef} (0.57,0.19,0.19,0.05), counter-based "
                           "generator seed 5, symmetrised, deduplicated, no loops; k-core (1,2)")
    if name.startswith("chunglu_n") and "_planted" in name:
        # chunglu_n{n}_g2.1_d20_planted{count}
        n = int(name.split("_n")[1].split("_")[0])
        count = int(name.split("_planted")[1])
        s1, d1 = chung_lu(n, 2.1, 20.0, seed=3)
        s2, d2 = plant_cliques(n, count, 20, 60, seed=3 + 1000)
        rp, col = to_csr(n, np.concatenate([s1, s2]), np.concatenate([d1, d2]))
        return dict(name=name, r=3, s=4, row_ptr=rp, col=col,
                    recipe=f"Chung-Lu n={n} gamma=2.1 mean degree 20 seed 3 plus {count} planted "
                           "cliques of size U[20,60] on random vertex sets; (3,4)-nucleus")
    raise KeyError(name)

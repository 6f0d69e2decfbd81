"""Planted mistakes in the oracle: every one must fail at least one pin.

Each mutant below is one plausible slip in ``oracle/oracle.c``: a flipped
comparison, a dropped term, a transposed operand, a wrong index, a missing
check.  For each, the oracle package is copied into a temporary directory,
the slip is applied to the copy's C source, and every pin of
``test_oracle_pins.py`` runs against the copy in a child process (so a
mutant that crashes cannot take the test run down).  The unmutated copy must
pass every pin; every mutant must fail at least one.  This is what shows the
pins constrain the oracle rather than merely agree with it.

Mutants that change nothing observable (for example a merge that skips one
side after a match, which the next comparison repairs) are left out: no pin
can tell them apart from the original.
"""
import concurrent.futures as cf
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")
ORACLE = os.path.join(ROOT, "oracle")

# name -> (text in oracle.c, replacement).  Each text occurs exactly once.
MUTANTS = {
    # Def. 3, the h-index
    "hindex_off_by_one": ("vals[h] >= h + 1) h++;", "vals[h] >= h) h++;"),
    "hindex_sorted_ascending": ("return (x < y) - (x > y);", "return (x > y) - (x < y);"),
    # Def. 4, rho = min over the other r-cliques of the s-clique
    "rho_max_not_min": ("if (src[S[k]] < rho) rho = src[S[k]];", "if (src[S[k]] > rho) rho = src[S[k]];"),
    "rho_drops_last_term": ("for (int k = 1; k < c->q; ++k) if (src[S[k]]",
                            "for (int k = 1; k < c->q - 1; ++k) if (src[S[k]]"),
    # tau_0 = d_s (Alg. 2 and Alg. 3 initialisation)
    "tau0_off_by_one": ("tau[R] = (int32_t)(c->inc_off[R + 1] - c->inc_off[R]);",
                        "tau[R] = (int32_t)(c->inc_off[R + 1] - c->inc_off[R] - 1);"),
    # Alg. 2: SND reads the previous pass, not the array being written
    "snd_reads_in_place": ("int32_t h = update_one(c, R, tp, L);\n            evals++;",
                           "int32_t h = update_one(c, R, tau, L);\n            evals++;"),
    "snd_stops_before_checking": ("        sweeps++;\n        if (!flag) break;\n        updating++;\n    }\nout:\n"
                                  "    if (sweeps_out) *sweeps_out = sweeps;\n    if (updating_out) *updating_out = updating;\n"
                                  "    if (evals_out) *evals_out = evals;\n    free(tp); free(L);",
                                  "        sweeps++;\n        updating++;\n        if (sweeps >= 1) break;\n    }\nout:\n"
                                  "    if (sweeps_out) *sweeps_out = sweeps;\n    if (updating_out) *updating_out = updating;\n"
                                  "    if (evals_out) *evals_out = evals;\n    free(tp); free(L);"),
    # Alg. 3 and the notification of Section 4.3
    "notify_strict": ("if (h <= tau[Rp] &&", "if (h < tau[Rp] &&"),
    "notify_skips_first_member": ("for (int k = 0; k < c->q; ++k) {\n                            int32_t Rp",
                                  "for (int k = 1; k < c->q; ++k) {\n                            int32_t Rp"),
    "notify_never_clears": ("                if (!act[R]) continue;\n                act[R] = 0;",
                            "                if (!act[R]) continue;"),
    "partial_updates_non_members": ("            if (members && !members[R]) continue;\n            if (notify) {",
                                    "            if (notify) {"),
    "partial_snd_updates_non_members": ("            if (!members[R]) continue;\n            int32_t h = update_one(c, R, tp, L);",
                                        "            int32_t h = update_one(c, R, tp, L);"),
    # Alg. 1, peeling
    "peel_decrements_equal_degree": ("if (d[Rp] > d[R]) {", "if (d[Rp] >= d[R]) {"),
    "peel_keeps_dead_s_cliques": ("if (skip) continue; /* an r-clique", "if (0 && skip) continue; /* an r-clique"),
    # Def. 5, degree levels
    "levels_double_count_shared_s_cliques": ("if (!ok || !owner) continue;", "if (!ok) continue;"),
    "levels_min_off_by_one": ("if (alive[R] && d[R] == mn) {", "if (alive[R] && d[R] <= mn + 1) {"),
    # Def. 1, the s-cliques of an r-clique
    "merge_advances_wrong_side": ("if (a < b) i++;\n        else if (b < a) j++;",
                                  "if (a < b) j++;\n        else if (b < a) i++;"),
    "k4_fourth_vertex_above_w_only": ("if (x == w || !adjacent(c, w, x)) continue;",
                                      "if (x <= w || !adjacent(c, w, x)) continue;"),
    "triangle_search_off_by_one": ("if (c->tri_w[mid] < x) lo = mid + 1; else hi = mid;",
                                   "if (c->tri_w[mid] <= x) lo = mid + 1; else hi = mid;"),
    "k4_drops_adjacency_test": ("if (x == w || !adjacent(c, w, x)) continue;", "if (x == w) continue;"),
    "tri_incidence_repeats_operand": ("buf[2 * i + 1] = (int32_t)b;", "buf[2 * i + 1] = (int32_t)a;"),
    "k4_incidence_wrong_triangle": ("d = tri_id(c, v, w, x);", "d = tri_id(c, u, w, x);"),
    "edge_tuples_transposed": ("out[2 * e] = c->eu[e]; out[2 * e + 1] = c->ev[e];",
                               "out[2 * e] = c->ev[e]; out[2 * e + 1] = c->eu[e];"),
    # input validation (Section 2: simple undirected graph)
    "accepts_unsorted_rows": ("if (p > rp[u] && col[p - 1] >= v) return ORC_E_INVAL;", ""),
    "accepts_self_loops": ("if (v < 0 || v >= n || v == u) return ORC_E_INVAL;",
                           "if (v < 0 || v >= n) return ORC_E_INVAL;"),
    "accepts_asymmetric": ("if (tc[p] != col[p]) st = ORC_E_INVAL;", ""),
    "symmetry_ignores_row_lengths": ("if (tp[v] != rp[v]) st = ORC_E_INVAL;", ""),
    # Kendall's tau-b (Section 5.2)
    "kendall_ties_transposed": ("tx += (sx == 0);", "tx += (sy == 0);"),
    "kendall_denominator_repeats_x": ("(n0 - (double)tx) * (n0 - (double)ty)", "(n0 - (double)tx) * (n0 - (double)tx)"),
    "kendall_counts_self_pairs": ("for (int64_t j = i + 1; j < n; ++j) {", "for (int64_t j = i; j < n; ++j) {"),
    "kendall_drops_sign_of_y": ("S += sx * sy;", "S += sx;"),
}

# Runs every pin of test_oracle_pins.py (slow ones excluded) against the
# oracle package found first on sys.path; prints the failing pins as JSON.
RUNNER = r"""
import inspect, json, sys
mut_dir, root, tests = sys.argv[1:4]
sys.path[:0] = [mut_dir, root, tests]
import oracle
assert oracle.__file__.startswith(mut_dir), oracle.__file__
import pytest
import test_oracle_pins as P
failed = []
for name, fn in inspect.getmembers(P, inspect.isfunction):
    if not name.startswith("test_"):
        continue
    marks = getattr(fn, "pytestmark", [])
    if any(m.name == "slow" for m in marks):
        continue
    cases = [{}]
    for m in marks:
        if m.name == "parametrize":
            names = m.args[0].split(",") if isinstance(m.args[0], str) else list(m.args[0])
            names = [x.strip() for x in names]
            cases = [dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]]
    for kw in cases:
        try:
            fn(**kw)
        except pytest.skip.Exception:
            pass
        except (Exception, pytest.fail.Exception) as e:
            failed.append("%s%s: %s" % (name, kw or "", type(e).__name__))
            break
print(json.dumps(failed))
"""


def _run(name, workdir):
    """Copy the oracle with one mutant applied (name None = unmutated) and run
    the pins against it.  Returns (exit code, failing pins or None)."""
    with open(os.path.join(ORACLE, "oracle.c")) as f:
        src = f.read()
    if name is not None:
        old, new = MUTANTS[name]
        assert src.count(old) == 1, f"{name}: the mutated text must occur exactly once"
        src = src.replace(old, new)
    mut_dir = os.path.join(workdir, name or "unmutated")
    pkg = os.path.join(mut_dir, "oracle")
    os.makedirs(pkg)
    shutil.copy(os.path.join(ORACLE, "__init__.py"), pkg)
    shutil.copy(os.path.join(ORACLE, "snd_mt.c"), pkg)
    with open(os.path.join(pkg, "oracle.c"), "w") as f:
        f.write(src)
    p = subprocess.run([sys.executable, "-c", RUNNER, mut_dir, ROOT, TESTS], capture_output=True,
                       text=True, timeout=300, cwd=mut_dir)
    lines = p.stdout.strip().splitlines()
    failed = json.loads(lines[-1]) if p.returncode == 0 and lines else None
    return p.returncode, failed, p.stderr[-2000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the mutated oracles")
    workdir = str(tmp_path_factory.mktemp("mutants"))
    names = [None] + sorted(MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        outs = list(ex.map(lambda nm: _run(nm, workdir), names))
    return dict(zip(names, outs))


def test_unmutated_copy_passes_every_pin(results):
    rc, failed, err = results[None]
    assert rc == 0 and failed == [], (rc, failed, err)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(results, name):
    rc, failed, err = results[name]
    # a crash (nonzero exit) also counts as caught: the pin run would fail
    assert rc != 0 or failed, f"mutant {name} passed every pin"

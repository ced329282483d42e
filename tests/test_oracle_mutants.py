"""The oracle's pins catch plausible mistakes in it.  Each mutant is a copy of the oracle's C source
with one planted mistake (a flipped comparison, a dropped term, a wrong constant, a skipped
guard), compiled into a temporary library and swapped in for the real one; the pin battery (brute
force, closed forms, worked examples, the threshold table against exact arithmetic) must fail on
every mutant and pass on the real oracle.  CPU only; nothing here touches the CUDA path."""
import os
import shutil
import subprocess
import sys

import pytest

import oracle
import test_oracle as pins

ORACLE_DIR = os.path.dirname(oracle.__file__)

# (name, exact snippet of nucleus_oracle.c, its replacement).  A mutation that cannot change any
# result is no test of the pins and is left out: e.g. letting Alg. 5 replace L[Q] by R when
# ND[L[Q]] == ND[R] (instead of linking R with L[Q]) joins the same components either way.
MUTANTS = [
    ("peel: decrement members already at the removed level",
     "if (u == R || d[u] <= d[R]) continue;", "if (u == R || d[u] < d[R]) continue;"),
    ("peel: an s-clique dies more than once",
     "      if (dead[S]) continue;\n      dead[S] = 1;\n      for (int j = 0; j < C; j++) {\n        int64_t u",
     "      dead[S] = 1;\n      for (int j = 0; j < C; j++) {\n        int64_t u"),
    ("hierarchy: s-clique joined at its largest member core",
     "for (int j = 1; j < C; j++) if (core[mem[j]] < core[mem[jmin]]) jmin = j;",
     "for (int j = 1; j < C; j++) if (core[mem[j]] > core[mem[jmin]]) jmin = j;"),
    ("r-subsets: repeated vertex in a subset",
     "for (int j = i + 1; j < r; j++) idx[j] = idx[j - 1] + 1;",
     "for (int j = i + 1; j < r; j++) idx[j] = idx[j - 1] + (j > 1);"),
    ("Alg. 2: bucket ends grow by (1 + delta/2)",
     "    x = x * (1.0 + delta);\n  }\n  return k;", "    x = x * (1.0 + 0.5 * delta);\n  }\n  return k;"),
    ("Alg. 2: first bucket end without the (1 + delta) factor",
     "double x = ((double)C + delta) * (1.0 + delta);", "double x = ((double)C + delta);"),
    ("Alg. 2: round cap without its + 1",
     "return (uint32_t)ceil(log(nn) / log1p(delta / (double)C)) + 1u;",
     "return (uint32_t)ceil(log(nn) / log1p(delta / (double)C));"),
    ("Alg. 2: value is the bucket end, not min(bucket end, degree)",
     "res->approx[R] = ti < cnt0[R] ? ti : cnt0[R];", "res->approx[R] = ti;"),
    ("Alg. 5: unequal levels united",
     "if (st->ND[R] == st->ND[Q]) {", "if (st->ND[R] <= st->ND[Q]) {"),
    ("Alg. 5: the walk down L[Q] stops early",
     "    } else {\n      lk_link(st, R, st->L[Q], depth + 1);\n      return;\n    }",
     "    } else {\n      return;\n    }"),
    ("construct-tree: single-leaf nodes kept",
     "if (root[C] == C && !(own[C] == 1 && nch[C] == 0)) nid[C] = nn++;", "if (root[C] == C) nid[C] = nn++;"),
]


def battery():
    """The pins of test_oracle.py that every mutant must fail at least once."""
    for r, s in [(1, 3), (2, 3), (2, 4), (3, 4), (2, 5)]:
        pins.test_oracle_vs_brute_force(r, s)
    for n, r, s in [(5, 2, 3), (6, 3, 4), (10, 2, 4), (9, 3, 5)]:
        pins.test_complete_graph_closed_form(n, r, s)
    pins.test_disjoint_planted_cliques()
    pins.test_two_k4_bridge_golden()
    pins.test_level_and_link_hierarchies_agree_medium()
    pins.test_link_efficient_worked_trace()
    pins.test_construct_tree_worked_trace()
    pins.test_approx_thresholds_closed_form()
    pins.test_approx_round_cap_formula()
    pins.test_approx_hand_worked_example()
    pins.test_approx_special_cases()


TESTS_DIR = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS_DIR)

# runs the battery against the library at argv[1] in a child process: a planted mistake may make
# the oracle fail an assertion, report an error or crash outright; any of them is "caught"
CHILD = """
import sys
sys.path[:0] = [{tests!r}, {root!r}]
import oracle
oracle._lib = None
oracle.build = lambda force=False: sys.argv[1]
import test_oracle_mutants
test_oracle_mutants.battery()
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_real_oracle_passes_the_battery():
    battery()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE_DIR, "nucleus_oracle.c")).read()
    assert src.count(old) == 1, "the mutation site must occur exactly once"
    mut = tmp_path / "nucleus_oracle.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-pthread", "-shared", "-fPIC", "-o", str(lib), str(mut),
                           os.path.join(ORACLE_DIR, "certify.c"), "-lm"])
    child = subprocess.run([sys.executable, "-c", CHILD.format(tests=TESTS_DIR, root=ROOT), str(lib)],
                           capture_output=True, text=True, timeout=600)
    assert child.returncode != 0, "no pin caught: " + name

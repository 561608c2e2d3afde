"""The oracle's pins must catch plausible mistakes.  Each case below plants one
mistake in a private copy of the oracle's C source (a dropped term, a wrong
comparison, a skipped check, an off-by-one), builds it on the CPU, and runs
the pin battery of ``test_oracle`` against it; at least one pin must fail."""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle as T

SRC = os.path.join(os.path.dirname(oracle.__file__), "truss_oracle.c")

MUTANTS = {
    "peel_decrements_at_equal_support": ("if (s <= k) return;", "if (s < k) return;"),
    "peel_ignores_removed_first_edge": ("if (w == y || removed[f1]) continue;", "if (w == y) continue;"),
    "peel_ignores_removed_second_edge": ("if (f2 < 0 || removed[f2]) continue;", "if (f2 < 0) continue;"),
    "trussness_offset": ("tau[e] = S[e] + 2;", "tau[e] = S[e] + 1;"),
    "support_skips_first_neighbour": (
        "for (int64_t j = g->off[a]; j < g->off[a + 1]; j++)\n        if (find_edge",
        "for (int64_t j = g->off[a] + 1; j < g->off[a + 1]; j++)\n        if (find_edge"),
    "canonical_keeps_repeats": ("if (i > 0 && key[i] == key[i - 1]) continue; /* repeated pair */", ""),
    "search_skips_entries": ("if (y < w) lo = mid + 1; else hi = mid - 1;",
                             "if (y < w) lo = mid + 2; else hi = mid - 1;"),
    "sublevel_only_case_ii_printed": (
        "if (S[e3] > l && (!(flag[e2] & F_INCURR) || e1 < e2)) {", "if (0) {"),
    "sublevel_without_tie_rule": ("(!(flag[e3] & F_INCURR) || e1 < e3)", "1"),
    "sublevel_ignores_processed": (
        "if ((flag[e2] & F_PROCESSED) || (flag[e3] & F_PROCESSED)) continue;", ""),
    "sublevel_next_on_wrong_value": ("if (S[e2] == l) next[nnext++] = e2;",
                                     "if (S[e2] == l + 1) next[nnext++] = e2;"),
    "sublevel_swapped_edge_roles": ("int32_t e2 = (a == v) ? f_aw : f_bw;", "int32_t e2 = (a == u) ? f_aw : f_bw;"),
    "components_hook_smaller_under_larger": ("if (a < b) p[b] = a;\n        else if (b < a) p[a] = b;",
                                             "if (a < b) p[a] = b;\n        else if (b < a) p[b] = a;"),
    "components_keep_low_trussness_edges": ("        if (tau[e] < k) continue;\n        const int32_t a",
                                            "        const int32_t a"),
}


def _battery():
    yield T.test_fig2_diamond
    yield T.test_complete_graphs
    yield T.test_fig1_caption_standin
    for c in T._fig3_cases():
        yield lambda c=c: T.test_fig3_sublevel_states(c)
    yield T.test_canonical_matches_set_definition
    yield T.test_random_graphs_up_to_14_vertices
    yield T.test_sublevel_frontiers_are_order_free
    yield T.test_all_graphs_on_six_vertices
    yield T.test_ktruss_components_closed_forms
    yield T.test_ktruss_components_match_connected_components


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    path_c = tmp_path / "mut.c"
    path_c.write_text(src.replace(old, new))
    path_so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                           str(path_c), "-o", str(path_so)])
    oracle.use_library(oracle.bind(str(path_so)))
    caught = None
    try:
        for check in _battery():
            try:
                check()
            except (AssertionError, ValueError, RuntimeError, MemoryError, IndexError) as ex:
                caught = ex
                break
    finally:
        oracle.use_library(None)
    assert caught is not None, f"no pin caught the planted mistake {name}"


def test_unmutated_copy_passes_battery(tmp_path):
    path_so = tmp_path / "libsame.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", SRC, "-o", str(path_so)])
    oracle.use_library(oracle.bind(str(path_so)))
    try:
        for check in _battery():
            check()
    finally:
        oracle.use_library(None)
    assert np.array_equal(oracle.truss(3, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32)), [3, 3, 3])

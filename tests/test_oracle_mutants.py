"""Plant plausible slips in copies of the oracle and check that the pins catch them.

Each mutant is oracle.c with one textual change, compiled to a temporary
library and swapped in as the oracle's default library while a subset of
the pin tests runs.  A mutant that passes every pin would mean the pins
cannot tell that slip from the correct oracle.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
import test_oracle_pins as pins
import test_oracle_cc
import test_oracle_mis
import test_oracle_mcm

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "drop_last_product": ("for (int32_t p = colptr[j]; p < colptr[j + 1]; ++p) {\n      int32_t i = rowidx[p];\n      ++nmult;",
                          "for (int32_t p = colptr[j]; p + 1 < colptr[j + 1]; ++p) {\n      int32_t i = rowidx[p];\n      ++nmult;"),
    "min_flipped": ("} else if (t < s->vi[i]) {", "} else if (t > s->vi[i]) {"),
    "mask_polarity": ("if (complement ? in_mask : !in_mask) continue;",
                      "if (complement ? !in_mask : in_mask) continue;"),
    "sum_sign": ("s->vd[i] += t;", "s->vd[i] -= t;"),
    "select1st": ("int32_t t = ((const int32_t*)x_val)[k]; /* select2nd",
                  "int32_t t = j; /* select2nd"),
    "bfs_level_off_by_one": ("      level[i] = L;\n      parent[i] = yv[q];",
                             "      level[i] = L + 1;\n      parent[i] = yv[q];"),
    "bfs_parent_self": ("      parent[i] = yv[q];", "      parent[i] = i;"),
    "cc_root_not_min": ("  for (int32_t v = 0; v < n; ++v) label[v] = low[uf_find(up, v)];",
                        "  for (int32_t v = 0; v < n; ++v) label[v] = uf_find(up, v);"),
    "cc_drops_last_edge": ("    for (int32_t p = colptr[j]; p < colptr[j + 1]; ++p) {\n      const int32_t i = rowidx[p];",
                           "    for (int32_t p = colptr[j]; p + 1 < colptr[j + 1]; ++p) {\n      const int32_t i = rowidx[p];"),
    "mis_descending_order": ("  return (pa > pb) - (pa < pb);", "  return (pa < pb) - (pa > pb);"),
    "mis_drops_last_neighbour": ("    for (int32_t p = colptr[v]; p < colptr[v + 1]; ++p) {\n      const int32_t u = rowidx[p];",
                                 "    for (int32_t p = colptr[v]; p + 1 < colptr[v + 1]; ++p) {\n      const int32_t u = rowidx[p];"),
    "mis_ignores_members": ("      if (u != v && in_set[u]) {", "      if (u != v && !in_set[u]) {"),
    "mcm_no_descent": ("      ++depth;  /* continue the alternating path through the column matched to row i */\n      scol[depth] = mate_r[i];\n      spos[depth] = colptr[mate_r[i]];",
                       "      continue;"),
    "mcm_skips_last_row": ("      if (p == colptr[j + 1]) {  /* every row of column j tried: back up */",
                           "      if (p + 1 >= colptr[j + 1]) {  /* every row of column j tried: back up */"),
    "mcm_flip_keeps_found": ("      mate_r[i] = j;\n      i = old;", "      mate_r[i] = j;\n      i = old >= 0 ? found : old;"),
    "mult_count_after_mask": ("      ++nmult; /* every selected column entry is one multiplication */\n      if (mask) {\n        int in_mask = mask[i] != 0;\n        if (complement ? in_mask : !in_mask) continue;\n      }",
                              "      if (mask) {\n        int in_mask = mask[i] != 0;\n        if (complement ? in_mask : !in_mask) continue;\n      }\n      ++nmult;"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    c = tmp_path / (name + ".c")
    c.write_text(src)
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so)])
    return oracle.load_variant(str(so))


def run_pins():
    """A fast subset of the pins; returns the names of the pins that failed."""
    failed = []
    checks = [
        ("dense_pt", lambda: pins.test_dense_closed_form(oracle.PLUS_TIMES, (33, 64), 0.3, "complement")),
        ("dense_min", lambda: pins.test_dense_closed_form(oracle.MIN_SELECT2ND, (64, 17), 0.3, "structural")),
        ("dense_bool", lambda: pins.test_dense_closed_form(oracle.OR_AND, (7, 5), 0.9, "none")),
        ("bruteforce", pins.test_bruteforce_all_subsets),
        ("mult_count", pins.test_multiply_count_invariant),
        ("bfs", lambda: pins.test_bfs_against_queue_bfs_and_scipy(*pins.GRAPHS[0])),
        ("grid", pins.test_intact_grid_levels_are_manhattan_distance),
        ("cc_hand", test_oracle_cc.test_hand_graph),
        ("cc_scipy", lambda: test_oracle_cc.test_against_scipy_and_invariants(2000, 3000, 5, 2)),
        ("mis_path", test_oracle_mis.test_path),
        ("mis_luby", lambda: test_oracle_mis.test_against_luby_rounds(400, 1600, 2)),
        ("mcm_greedy_undone", test_oracle_mcm.test_first_greedy_choice_must_be_undone),
        ("mcm_scipy", lambda: test_oracle_mcm.test_against_scipy_hopcroft_karp(1000, 1500, 2200, 2)),
    ]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError):
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_the_subset():
    assert run_pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    lib = build_mutant(tmp_path, name)
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = run_pins()
    assert failed, "mutant %s passed every pin" % name

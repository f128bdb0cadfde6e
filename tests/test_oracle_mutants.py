"""Planted mistakes in a private copy of the oracle must each fail at least one pin.

This shows the pins are tight enough to catch a dropped term, a wrong index, a
wrong scale factor or a mis-ordered update anywhere in the oracle.  The copy
is compiled into a temporary directory on the CPU; the real oracle is untouched.
"""
import os
import subprocess

import pytest

import oracle as O
import oracle_pins as P

MUTANTS = {
    "drop_local_w": ("if (l_sum) l_sum[w] += 1;", ""),
    "local_v_dropped": ("if (l_sum) { l_sum[u] += nuv; l_sum[v] += nuv; }", "if (l_sum) { l_sum[u] += nuv; }"),
    "groups_share_seed": ("(uint64_t)k * 0x9E3779B97F4A7C15ULL", "(uint64_t)0"),
    "splitmix_shift": ("return z ^ (z >> 31);", "return z ^ (z >> 32);"),
    "store_wrong_colour": ("if (orc_colour(u, v, seed, k, m) == j) {", "if (orc_colour(u, v, seed, k, m) <= j) {"),
    "slot_index_off_by_one": ("*j = mascot ? 0 : i % m;", "*j = mascot ? 0 : (i + 1) % m;"),
    "scale_m_over_c": ("double f = md * md / (double)c;", "double f = md / (double)c;"),
    "scale_full_groups": ("double f1 = md / (double)c1;", "double f1 = md * md / (double)c1;"),
    "pair_counter_starts_at_nuv": ("edge_key(u, v), 0);", "edge_key(u, v), nuv);"),
    "eta_local_u_uses_vw": ("eta_local[u] += *tuw;", "eta_local[u] += *tvw;"),
    "static_last_edge_wrong": ("if (e[q] > e[last]) last = q;", "if (e[q] < e[last]) last = q;"),
    "mascot_samplers_share_hash": ("*k = mascot ? i : i / m;", "*k = mascot ? 0 : i / m;"),
    "mascot_keeps_colour_i": ("*j = mascot ? 0 : i % m;", "*j = mascot ? i % m : i % m;"),
    "mascot_scale_p_not_p2": ("double inv_p2 = md * md;", "double inv_p2 = md;"),
    "local_weights_swapped": ("est_local[v] = (v1 + v2 > 0.0) ? (v2 * a1 + v1 * a2) / (v1 + v2) : a1;",
                              "est_local[v] = (v1 + v2 > 0.0) ? (v1 * a1 + v2 * a2) / (v1 + v2) : a1;"),
    "local_eta_scaled_m2": ("double eh = (double)eta_local[v] * (md * md * md / (double)c);",
                            "double eh = (double)eta_local[v] * (md * md / (double)c);"),
    "local2_scale_full_groups": ("double a1 = (double)local1[v] * f1, a2 = (double)local2[v] * f2;",
                                 "double a1 = (double)local1[v] * f1, a2 = (double)local2[v] * f1;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(O._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "rept_oracle_mutant.c"
    path.write_text(src.replace(old, new))
    lib_path = str(tmp_path / f"librept_oracle_{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", str(path), "-o", lib_path])
    lib = O.load_library(lib_path)
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(lib=lib)
        except AssertionError:
            failed.append(pin.__name__)
            break
    assert failed, f"planted mistake {name} passed every pin"

"""Plants plausible mistakes in a temporary copy of the oracle (on the CPU) and checks that the pins
of test_oracle.py catch every one of them: a dropped term, a wrong index or sign, a transposed
operand, a batch that reads its own new values, a broken permutation, a wrong tie-break.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as obuild
import test_oracle as T

SRC = os.path.join(os.path.dirname(obuild.__file__), "oracle.c")

MUTANTS = {
    "drop_discount": ("return g + M->gamma * acc;", "return g + acc;"),
    "wrong_successor_index": ("acc += (double)M->prob[e] * J[M->col[e]];",
                              "acc += (double)M->prob[e] * J[M->col[M->row_ptr[r]]];"),
    "transposed_dense_row": ("const float *row = M->P + r * M->n;",
                             "const float *row = M->P + ((int64_t)a * M->n + s) * M->n;"),
    "batch_reads_own_new_values": (
        "            if (pi) W[i] = orc_q(M, s, pi[s], V);\n            else    W[i] = backup_min(M, s, V, NULL, NULL);",
        "            if (pi) W[i] = orc_q(M, s, pi[s], V);\n            else    W[i] = backup_min(M, s, V, NULL, NULL);\n            V[s] = W[i];"),
    "batch_boundary_off_by_one": ("for (int64_t start = 0; start < n; start += b) {",
                                  "for (int64_t start = 0; start < n; start += (b > 1 ? b - 1 : b)) {"),
    "feistel_wrong_xor": ("uint64_t newR = L ^ F;", "uint64_t newR = R ^ F;"),
    "philox_swapped_multipliers": ("uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;",
                                   "uint64_t prod0 = (uint64_t)PHILOX_M1 * (uint64_t)x0;"),
    "argmin_ties_to_highest": ("if (q < best) { second = best; best = q; ba = a; }",
                               "if (q <= best) { second = best; best = q; ba = a; }"),
    "mpi_evaluates_wrong_policy_rows": ("            apply_order(M, pi, b, perm, V, W);\n            sweep++;",
                                        "            apply_order(M, NULL, b, perm, V, W);\n            sweep++;"),
    "weighted_search_off_by_one": ("if (cum[mid] > r) hi = mid;", "if (cum[mid] >= r) hi = mid;"),
    "draws_reuse_the_feistel_stream": ("uint32_t ctr[4] = { (uint32_t)p, 0x80000000u,", "uint32_t ctr[4] = { (uint32_t)p, 0u,"),
    "weights_ignored": ("        run += w[s];", "        run += 1;"),
    "stop_without_full_residual": ("            resid = full_residual(M, pi, V);\n            if (resid <= eps) break;",
                                   "            break;"),
    "delta_not_a_change": ("double d = fabs(W[i] - V[s]);", "double d = fabs(W[i]);"),
}

PINS = [
    T.test_philox_known_answers,
    lambda: T.test_perm_is_bijection(5),
    lambda: T.test_perm_is_bijection(500),
    T.test_golden_two_state_closed_form,
    lambda: T.test_mbvi_matches_brute_force(0),
    lambda: T.test_mbvi_matches_brute_force(1),
    lambda: T.test_policy_evaluation_closed_form(1),
    lambda: T.test_mb_apply_matches_set_definition(0),
    lambda: T.test_mb_apply_matches_set_definition(1),
    T.test_reductions_b_equals_n_and_b_equals_1,
    T.test_delta_is_sup_norm_change,
    T.test_mpi_first_outer_iteration_closed_form,
    T.test_mpi_matches_policy_iteration,
    T.test_greedy_ties_resolve_to_lowest_action,
    T.test_draws_follow_their_definition,
    T.test_constant_weights_reproduce_uniform_draws,
    lambda: T.test_with_replacement_sweep_matches_definition(1),
    T.test_with_replacement_converges_under_the_stop_rule,
    T.test_bellman_residual_stop_rule,
]


def _build_mutant(tmp, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = os.path.join(tmp, "mut.c")
    open(path, "w").write(src.replace(old, new))
    so = os.path.join(tmp, "libmut.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", so, path, "-lm"],
                   check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    old, new = MUTANTS[name]
    tmp = tempfile.mkdtemp(prefix="orc_mut_")
    try:
        so = _build_mutant(tmp, old, new)
        real = oracle.lib()
        mut = ctypes.CDLL(so)
        for fn in ("orc_philox4x32_10", "orc_perm", "orc_perm_all", "orc_perm_half_bits", "orc_q",
                   "orc_greedy", "orc_mb_apply", "orc_mbvi", "orc_mpi", "orc_bellman_T",
                   "orc_gauss_seidel_F", "orc_num_threads", "orc_sweep_order", "orc_mbvi_select",
                   "orc_mpi_select"):
            f, g = getattr(mut, fn), getattr(real, fn)
            f.argtypes, f.restype = g.argtypes, g.restype
        monkeypatch.setattr(oracle, "_LIB", mut)
        oracle._BOUND_CACHE.clear()
        caught = []
        for pin in PINS:
            try:
                pin()
            except (AssertionError, RuntimeError, ValueError, IndexError):
                caught.append(pin)
                break
        assert caught, f"no pin caught the planted mistake {name}"
    finally:
        oracle._BOUND_CACHE.clear()
        shutil.rmtree(tmp, ignore_errors=True)


# Planted mistakes in a copy of exact.py's dense certificate (the FP64 policy iteration used on the
# n = 16384 dense workload), each caught by one of its pins.
EXACT_MUTANTS = {
    "dense_pass_drops_discount": ("Q[s0:s1] = c[s0:s1] + gamma * (R @ J).reshape(s1 - s0, m)",
                                  "Q[s0:s1] = c[s0:s1] + (R @ J).reshape(s1 - s0, m)"),
    "dense_pass_wrong_chunk_rows": ("R = np.asarray(rows_of(s0 * m, s1 * m), dtype=np.float64)",
                                    "R = np.asarray(rows_of(s0, s1 * m - s0 * (m - 1)), dtype=np.float64)"),
    "policy_solve_transposed": ("        J = np.linalg.solve(A, g)\n        del A",
                                "        J = np.linalg.solve(A.T, g)\n        del A"),
    "policy_rows_of_the_wrong_action": ("A = np.asarray(rows_at(states * m + pi), dtype=np.float64)",
                                        "A = np.asarray(rows_at(states * m + (pi + 1) % m), dtype=np.float64)"),
    "improvement_takes_the_maximum": ("new_pi = np.where(keep, pi, np.argmin(Q, axis=1))",
                                      "new_pi = np.where(keep, pi, np.argmax(Q, axis=1))"),
}

EXACT_PINS = [T.test_dense_policy_iteration_matches_brute_force, T.test_dense_policy_iteration_matches_converged_mbvi,
              T.test_dense_bellman_pass_matches_the_oracle]


@pytest.mark.parametrize("name", sorted(EXACT_MUTANTS))
def test_pins_catch_planted_mistake_in_the_dense_certificate(name):
    import importlib.util
    old, new = EXACT_MUTANTS[name]
    src = open(os.path.join(os.path.dirname(obuild.__file__), "exact.py")).read()
    assert src.count(old) == 1, old
    tmp = tempfile.mkdtemp(prefix="exact_mut_")
    try:
        path = os.path.join(tmp, "exact_mut.py")
        open(path, "w").write(src.replace(old, new))
        spec = importlib.util.spec_from_file_location("exact_mut", path)
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        caught = False
        for pin in EXACT_PINS:
            try:
                pin(ex=mod)
            except (AssertionError, RuntimeError, ValueError, IndexError, np.linalg.LinAlgError):
                caught = True
                break
        assert caught, f"no pin caught the planted mistake {name}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)

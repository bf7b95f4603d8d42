"""The pins are strong enough: plant a plausible mistake in one oracle step (on the CPU)
and check that at least one pin of ``test_oracle_pins`` fails."""
import numpy as np
import pytest

import oracle.odmd_ref as ref
from tests import test_oracle_pins as pins

PIN_FUNCS = [
    lambda: pins.test_incremental_equals_batch_without_truncation(64, 12, 1),
    pins.test_reduced_operator_equals_definition,
    pins.test_planted_modes_noise_free_recovers_eigenvalues,
    pins.test_linear_system_one_step_identity,
    pins.test_rollout_matches_analytic_stream,
    pins.test_truncation_bound_and_orthonormality,
    pins.test_check_special_cases,
]


def _mutations():
    orig_op = ref.operator_update
    orig_rows = ref.right_rows_update
    orig_rot = ref.rotate_basis
    orig_core = ref.core_matrix
    orig_dir = ref.new_direction
    orig_pow = ref.OnlineDMDRef.powers

    def op_sign(M, w, rho, r_last, gamma, U1, V1):
        return orig_op(M, w, -rho, r_last, gamma, U1, V1)

    def op_drop_w(M, w, rho, r_last, gamma, U1, V1):
        return orig_op(M, 0 * w, rho, r_last, gamma, U1, V1)

    def op_swap(M, w, rho, r_last, gamma, U1, V1):
        return orig_op(M, w, rho, r_last, gamma, V1, U1)

    def rows_index(r_first, V1):
        rf, _ = orig_rows(r_first, V1)
        return rf, V1[0, :].copy()

    def rows_first(r_first, V1):
        _, rl = orig_rows(r_first, V1)
        return np.append(r_first, 1.0) @ V1, rl

    def rot_transposed(L, j, U1):
        if U1.shape[0] == U1.shape[1]:
            return orig_rot(L, j, U1.T)
        return orig_rot(L, j, U1[:, ::-1])

    def core_transposed(S, p, rho):
        return orig_core(S, p, rho).T

    def dir_unnormalised(e, sigma1, cnorm, tau):
        rho, j = orig_dir(e, sigma1, cnorm, tau)
        return rho, j * rho if rho > 0 else j

    def pow_shift(lam, t):
        return orig_pow(lam, t + 1.0)

    def gs_once(L, c, p):
        # classical Gram-Schmidt applied once: the correction s = L^T e is never taken
        return p, c - L @ p

    return [
        ("operator_update", op_sign),
        ("operator_update", op_drop_w),
        ("operator_update", op_swap),
        ("right_rows_update", rows_index),
        ("right_rows_update", rows_first),
        ("rotate_basis", rot_transposed),
        ("core_matrix", core_transposed),
        ("new_direction", dir_unnormalised),
        ("powers", staticmethod(pow_shift)),
        ("orthogonalise_cgs2", gs_once),
    ]


@pytest.mark.parametrize("idx", range(10))
def test_planted_mistake_is_caught(idx, monkeypatch):
    name, bad = _mutations()[idx]
    if name == "powers":
        monkeypatch.setattr(ref.OnlineDMDRef, "powers", bad)
    else:
        monkeypatch.setattr(ref, name, bad)
    failures = 0
    for f in PIN_FUNCS:
        try:
            with np.errstate(all="ignore"):
                f()
        except (AssertionError, np.linalg.LinAlgError, ValueError, IndexError, FloatingPointError):
            failures += 1
    assert failures >= 1, f"mutation {idx} ({name}) slipped through every pin"

"""The oracle's pins are sensitive: plant a plausible mistake in the oracle (on the
CPU, through monkeypatch) and check that at least one pin fails."""
import numpy as np
import pytest

import oracle
import oracle.fp64 as OL
import tests.test_oracle_pins as P


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(OL, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _fails(test, *args):
    with pytest.raises(AssertionError):
        test(*args)


def test_transposed_procrustes_is_caught(monkeypatch):
    good = OL.procrustes
    _patch(monkeypatch, "procrustes", lambda Zi, Zb: good(Zi, Zb).T)
    _fails(P.test_procrustes_lemma_identities)


def test_unweighted_average_is_caught(monkeypatch):
    # averaging with 1/m instead of p_i = s_i/n (uneven partitions)
    _patch(monkeypatch, "weights", lambda sizes: np.full(len(sizes), 1.0 / len(sizes)))
    _fails(P.test_p1_is_distributed_power_iteration, "sign")


def test_local_step_with_global_scale_is_caught(monkeypatch):
    # M_i formed with 1/n (wrong) while the average still weighs by s_i/n
    def bad(A_i, Z):
        A = OL.as_f64(A_i)
        return (A.T @ (A @ Z)) / 600.0
    _patch(monkeypatch, "local_step", bad)
    _fails(P.test_p1_is_distributed_power_iteration, "sign")


def test_orth_without_sign_convention_is_caught(monkeypatch):
    def bad(Y):
        Q, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64))
        return -Q
    _patch(monkeypatch, "orth", bad)
    _fails(P.test_orth_is_q_factor_with_positive_r_diagonal)


def test_sign_fix_on_wrong_columns_is_caught(monkeypatch):
    def bad(Zi, Zb):
        c = np.einsum("dj,dj->j", Zi, Zb[:, ::-1])
        return np.diag(np.where(c < 0, -1.0, 1.0))
    _patch(monkeypatch, "sign_fix", bad)
    _fails(P.test_sign_fix_is_the_brute_force_minimiser)


def test_smallest_partition_as_base_is_caught(monkeypatch):
    _patch(monkeypatch, "base_index", lambda sizes: int(np.argmin(np.asarray(sizes))))
    _fails(P.test_aggregation_invariances)


def test_aggregation_without_alignment_is_caught(monkeypatch):
    _patch(monkeypatch, "align", lambda kind, Zi, Zb: np.eye(Zi.shape[1]))
    _fails(P.test_aggregation_invariances)


def test_ritz_with_wrong_scale_is_caught(monkeypatch):
    good = OL.ritz

    def bad(parts, Z):
        Zr, s = good(parts, Z)
        return Zr, s / np.sqrt(len(parts))
    _patch(monkeypatch, "ritz", bad)
    _fails(P.test_ritz_recovers_singular_values)

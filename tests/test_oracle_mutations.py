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


def test_round_loop_that_ignores_the_aggregator_is_caught(monkeypatch):
    # the loop passes "identity" to the aggregation whatever the caller asked for
    good = OL.aggregate
    _patch(monkeypatch, "aggregate", lambda Y_loc, Z_loc, sizes, kind: good(Y_loc, Z_loc, sizes, "identity"))
    _fails(P.test_round_loop_matches_matrix_power_route, "sign")
    _fails(P.test_round_loop_matches_matrix_power_route, "opt")
    _fails(P.test_aggregators_differ_at_p_above_1)


def test_round_loop_that_aligns_the_wrong_basis_is_caught(monkeypatch):
    # the loop aligns orth(Y_i) (the basis after the last multiply) instead of the
    # basis Z_i that was multiplied (App. B: D_t aligns the iterate M_i was applied to)
    good = OL.aggregate
    _patch(monkeypatch, "aggregate",
           lambda Y_loc, Z_loc, sizes, kind: good(Y_loc, [OL.orth(Y) for Y in Y_loc], sizes, kind))
    _fails(P.test_round_loop_matches_matrix_power_route, "opt")


def test_ritz_with_wrong_scale_is_caught(monkeypatch):
    good = OL.ritz

    def bad(parts, Z):
        Zr, s = good(parts, Z)
        return Zr, s / np.sqrt(len(parts))
    _patch(monkeypatch, "ritz", bad)
    _fails(P.test_ritz_recovers_singular_values)


def _eta_variant(mean_weights=None, local_scale=None, signed=False, by_trace=False):
    """An eta with one planted mistake (Def. 2 is max_i ||M_i - M||_2 / ||M||_2)."""
    def bad(parts):
        As = [OL.as_f64(P_) for P_ in parts]
        sizes = [A.shape[0] for A in As]
        n = sum(sizes)
        p = OL.weights(sizes) if mean_weights is None else mean_weights(sizes)
        Ms = [A.T @ A / (A.shape[0] if local_scale is None else local_scale(n, A.shape[0])) for A in As]
        M = sum(pi * Mi for pi, Mi in zip(p, Ms))
        norm = (lambda X: float(np.max(np.linalg.eigvalsh(X)))) if signed else \
               (lambda X: float(np.max(np.abs(np.linalg.eigvalsh(X)))))
        norms = [norm(Mi - M) for Mi in Ms]
        den = float(np.trace(M)) if by_trace else norm(M)
        return max(norms) / den, np.array(norms + [den])
    return bad


@pytest.mark.parametrize("variant", [
    dict(mean_weights=lambda sizes: np.full(len(sizes), 1.0 / len(sizes))),   # unweighted M
    dict(local_scale=lambda n, s: n),                                        # M_i with 1/n
    dict(signed=True),                                                       # largest eigenvalue, not |.|
    dict(by_trace=True),                                                     # normalised by trace(M)
])
def test_eta_mistakes_are_caught(monkeypatch, variant):
    _patch(monkeypatch, "eta", _eta_variant(**variant))
    _fails(P.test_eta_closed_form_for_axis_aligned_partitions)


def test_residual_error_in_frobenius_norm_is_caught(monkeypatch):
    good_align = OL.align

    def bad(Z_loc, sizes, kind):
        b = OL.base_index(sizes)
        Zb = Z_loc[b]
        return max(float(np.linalg.norm(Z @ good_align(kind, Z, Zb) - Zb)) for i, Z in enumerate(Z_loc) if i != b)
    _patch(monkeypatch, "residual_error", bad)
    _fails(P.test_residual_error_with_opt_matches_the_procrustes_lemma)

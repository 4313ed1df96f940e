"""Pins for the FP64 oracle: each check compares it with something other than
itself (a closed form, a different algorithm, brute force, a library routine
used on a different formulation).  CPU only."""
import itertools

import numpy as np
import pytest

import oracle as O
import synth


def _rng(s):
    return np.random.default_rng(s)


def _orthonormal(d, k, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((d, k)))
    return Q


def _small_problem(seed=0, n=600, d=12, lam=(9.0, 5.0, 3.0, 1.0), sigma=0.3, sizes=(250, 200, 150)):
    A = synth.spiked_rows(n, d, np.array(lam), sigma, seed, out_dtype=np.float64, threads=1)
    parts = synth.split_rows(A, list(sizes))
    return A, parts


def _qr_power(M, Y0, steps):
    """orth(M^steps Y0) by one matrix power and one QR (a route the oracle never takes)."""
    Q, R = np.linalg.qr(np.linalg.matrix_power(M, steps) @ Y0)
    return Q * np.sign(np.diag(R))


# --------------------------------------------------------------------------- metric

def test_subspace_dist_matches_definition_and_angles():
    rng = _rng(1)
    for _ in range(20):
        d, k = 15, 4
        U, V = _orthonormal(d, k, rng), _orthonormal(d, k, rng)
        explicit = np.linalg.norm(U @ U.T - V @ V.T, 2)               # Def. 1 verbatim
        cos_min = np.linalg.svd(U.T @ V, compute_uv=False).min()      # cos theta_k
        assert O.subspace_dist(U, V) == pytest.approx(explicit, abs=1e-13)
        assert O.subspace_dist(U, V) == pytest.approx(np.sqrt(max(0.0, 1 - cos_min ** 2)), abs=1e-10)
    U = _orthonormal(10, 3, rng)
    assert O.subspace_dist(U, U @ _orthonormal(3, 3, rng)) < 1e-14     # same span
    E = np.eye(6)
    assert O.subspace_dist(E[:, :2], E[:, 2:4]) == pytest.approx(1.0)  # orthogonal spans


def test_subspace_dist_tiny_angle_accuracy():
    # A rotation by a known tiny angle theta in the (e1, e4) plane: dist = sin(theta).
    for theta in (1e-4, 1e-7, 1e-10):
        U = np.eye(8)[:, :3]
        V = U.copy()
        V[:, 0] = np.cos(theta) * np.eye(8)[:, 0] + np.sin(theta) * np.eye(8)[:, 3]
        assert O.subspace_dist(U, V) == pytest.approx(np.sin(theta), rel=1e-6)


# --------------------------------------------------------------------------- orth

def test_orth_is_q_factor_with_positive_r_diagonal():
    rng = _rng(2)
    Y = rng.standard_normal((40, 7)) @ np.diag([1e3, 1, 1, 1e-2, 5, 1, 1])
    Q = O.orth(Y)
    R = Q.T @ Y
    assert np.abs(Q.T @ Q - np.eye(7)).max() < 1e-14
    assert np.abs(np.tril(R, -1)).max() < 1e-10 * np.abs(R).max()
    assert (np.diag(R) > 0).all()
    assert np.abs(Q @ R - Y).max() < 1e-12 * np.abs(Y).max()


# --------------------------------------------------------------------------- whole loop

@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
def test_p1_is_distributed_power_iteration(agg):
    """p = 1 is DPI (Sec. 3, the special case below the definition of I_T): after T
    rounds the output spans M^T Z_0 with M = sum_i p_i M_i formed explicitly."""
    A, parts = _small_problem(seed=3)
    Y0 = synth.gaussian_start(12, 3, 5)
    T = 9
    r = O.localpower(parts, 3, [1] * T, agg, Y0)
    M = A.T @ A / A.shape[0]
    assert O.subspace_dist(r["Z"], _qr_power(M, Y0, T)) < 1e-10  # matrix power: cond ~ (lam1/lam3)^T
    assert r["rounds"] == T and r["local_steps"] == T


@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
def test_single_partition_is_subspace_iteration(agg):
    A, _ = _small_problem(seed=4, sizes=(600,))
    Y0 = synth.gaussian_start(12, 3, 6)
    sched = [3, 2, 4, 1]
    r = O.localpower([A], 3, sched, agg, Y0)
    M = A.T @ A / A.shape[0]
    assert O.subspace_dist(r["Z"], _qr_power(M, Y0, sum(sched))) < 1e-10


@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
def test_replicated_partitions_have_no_local_drift(agg):
    """eta = 0 (every M_i = M, Def. 2): local iterates never drift apart, so the
    output equals subspace iteration with sum(p_t) steps."""
    A, _ = _small_problem(seed=5, n=300, sizes=(300,))
    Y0 = synth.gaussian_start(12, 3, 7)
    sched = [4, 4, 2]
    r = O.localpower([A, A.copy(), A.copy()], 3, sched, agg, Y0)
    M = A.T @ A / A.shape[0]
    assert O.subspace_dist(r["Z"], _qr_power(M, Y0, sum(sched))) < 1e-10


@pytest.mark.parametrize("agg", ["sign", "opt"])
def test_decay_to_p1_converges_to_eigh(agg):
    """With p decayed to 1 the error goes to zero (Sec. 3, decaying p; Sec. 5):
    compare with a full eigendecomposition of M."""
    A, parts = _small_problem(seed=6, d=8, lam=(8.0, 6.0, 4.0), sigma=0.5, n=900, sizes=(400, 300, 200))
    Y0 = synth.gaussian_start(8, 3, 8)
    sched = [8] * 3 + [4] * 3 + [2] * 3 + [1] * 80
    r = O.localpower(parts, 3, sched, agg, Y0)
    lam, V = np.linalg.eigh(A.T @ A / A.shape[0])
    assert O.subspace_dist(r["Z"], V[:, -3:]) < 1e-10


def _heterogeneous_parts(seed, sizes=(250, 200, 150), d=12):
    """Uneven partitions drawn from different spiked models (each its own Haar
    rotation), so the local iterates drift far apart within a round and both
    sign-fixing and OPT have work to do (large eta, Def. 2)."""
    return [synth.spiked_rows(s, d, np.array((9.0, 5.0, 3.0, 1.0)), 0.3, seed * 10 + i,
                              out_dtype=np.float64, threads=1) for i, s in enumerate(sizes)]


def _polar_factor_newton(C, iters=60):
    """Orthogonal polar factor of a nonsingular C by the Newton iteration
    X <- (X + X^{-T}) / 2 (a route that uses no SVD).  For C = W1 S W2^T it
    converges to W1 W2^T, the minimiser of eq. (3)."""
    X = np.array(C, dtype=np.float64)
    for _ in range(iters):
        X = 0.5 * (X + np.linalg.inv(X).T)
    return X


def _sign_by_enumeration(Z_i, Z_b):
    """The +-1 diagonal D minimising ||Z_i D - Z_b||_F, by trying all 2^k of them (eq. (4))."""
    k = Z_i.shape[1]
    best = min(itertools.product((1.0, -1.0), repeat=k),
               key=lambda s: np.linalg.norm(Z_i * np.array(s) - Z_b))
    return np.diag(best)


def _round_by_matrix_powers(parts, Y, p, kind):
    """One round of Alg. 1 with the aligned aggregation of eqs. (3)-(4), built by a
    route the oracle never takes: every M_i is formed densely, the basis worker i
    multiplies in its last local step is orth(M_i^(p-1) Z) from one matrix power
    and one QR (the local iterate is the Q factor of the i-th matrix power times
    Z, Sec. 3), Y_i = M_i times that basis, the aligner comes from enumeration
    (signs) or a Newton polar iteration (OPT), and Y = sum_i (s_i/n) Y_i D_i with
    D_b = I for the largest partition b (App. B update rule)."""
    sizes = [P.shape[0] for P in parts]
    n = float(sum(sizes))
    b = sizes.index(max(sizes))
    Ms = [P.T @ P / P.shape[0] for P in parts]
    Z = _qr_power(np.eye(Y.shape[0]), Y, 0)
    last = [_qr_power(M, Z, p - 1) for M in Ms]
    out = np.zeros_like(Y)
    for i, (M, Zl) in enumerate(zip(Ms, last)):
        if i == b or p == 1 or kind == "identity":
            D = np.eye(Y.shape[1])
        elif kind == "sign":
            D = _sign_by_enumeration(Zl, last[b])
        else:
            D = _polar_factor_newton(Zl.T @ last[b])
        out += (sizes[i] / n) * (M @ Zl) @ D
    return out


@pytest.mark.parametrize("agg", ["identity", "sign", "opt"])
def test_round_loop_matches_matrix_power_route(agg):
    """The whole round loop at p > 1 with m = 3 uneven, heterogeneous partitions:
    the oracle's Y after T = 1, 2 and 3 rounds (schedule 3, 3, then a p = 1
    round that aggregates without alignment) equals the matrix-power route
    round by round, for all three aggregators."""
    parts = _heterogeneous_parts(6)
    Y0 = synth.gaussian_start(12, 3, 13)
    sched = [3, 3, 1]
    Y = Y0
    for T in range(1, len(sched) + 1):
        Y = _round_by_matrix_powers(parts, Y, sched[T - 1], agg)
        got = O.localpower(parts, 3, sched[:T], agg, Y0)["Y"]
        assert np.abs(got - Y).max() <= 1e-12 * np.abs(Y).max(), (agg, T)


def test_aggregators_differ_at_p_above_1():
    """With drifting local iterates the three update rules of App. B give three
    different aggregates (so a loop that ignores the aggregator is visible), and
    at p = 1 they coincide."""
    parts = _heterogeneous_parts(6)
    Y0 = synth.gaussian_start(12, 3, 13)
    Ys = {a: O.localpower(parts, 3, [3, 2], a, Y0)["Y"] for a in O.AGGREGATORS}
    scale = np.abs(Ys["identity"]).max()
    for a, c in (("identity", "sign"), ("identity", "opt"), ("sign", "opt")):
        assert np.abs(Ys[a] - Ys[c]).max() > 1e-2 * scale, (a, c)
    Y1 = {a: O.localpower(parts, 3, [1, 1], a, Y0)["Y"] for a in O.AGGREGATORS}
    assert max(np.abs(Y1[a] - Y1["identity"]).max() for a in O.AGGREGATORS) == 0.0


def test_constant_p_leaves_a_floor_that_p1_removes():
    """Sec. 5 (final precision): with a constant p > 1 the error stops decreasing at
    a non-zero floor; p = 1 does not have one.  Qualitative (the floor's value has
    no closed form: parity unpinned)."""
    A, parts = _small_problem(seed=7, d=10, lam=(5.0, 4.0, 3.0), sigma=0.6, n=200, sizes=(50, 50, 50, 50))
    Y0 = synth.gaussian_start(10, 3, 9)
    lam, V = np.linalg.eigh(A.T @ A / A.shape[0])
    truth = V[:, -3:]
    e1 = O.localpower(parts, 3, [1] * 120, "sign", Y0, truth=truth)["trace"][-1]["dist"]
    e8 = O.localpower(parts, 3, [8] * 60, "sign", Y0, truth=truth)
    assert e1 < 1e-8
    d8 = [t["dist"] for t in e8["trace"]]
    assert d8[-1] > 1e-4 and abs(d8[-1] - d8[-10]) < 1e-3 * d8[-1] + 1e-12


# --------------------------------------------------------------------------- alignment

def test_procrustes_lemma_identities():
    """App. A, Lemma (orthogonal Procrustes): ||U - U~ O*||_2 = sqrt(2 - 2 sqrt(1 - dist^2))
    and dist <= ||U - U~ O*||_2 <= sqrt(2) dist, with O* from the SVD of U~^T U."""
    rng = _rng(10)
    for scale in (1e-3, 1e-1, 0.5, 2.0):
        for _ in range(10):
            U = _orthonormal(20, 4, rng)
            Ut = O.orth(U @ _orthonormal(4, 4, rng) + scale * rng.standard_normal((20, 4)))
            Ostar = O.procrustes(Ut, U)
            dd = np.linalg.norm(U - Ut @ Ostar, 2)
            dist = O.subspace_dist(U, Ut)
            assert dd == pytest.approx(np.sqrt(2 - 2 * np.sqrt(1 - dist ** 2)), rel=1e-9, abs=1e-14)
            assert dist - 1e-12 <= dd <= np.sqrt(2) * dist + 1e-12
            assert np.abs(Ostar.T @ Ostar - np.eye(4)).max() < 1e-13


def test_procrustes_is_the_frobenius_minimiser():
    rng = _rng(11)
    Zi, Zb = _orthonormal(15, 3, rng), _orthonormal(15, 3, rng)
    best = np.linalg.norm(Zi @ O.procrustes(Zi, Zb) - Zb)
    for _ in range(500):
        Q = _orthonormal(3, 3, rng)
        assert best <= np.linalg.norm(Zi @ Q - Zb) + 1e-12


def test_sign_fix_is_the_brute_force_minimiser():
    rng = _rng(12)
    for _ in range(20):
        Zi, Zb = _orthonormal(9, 5, rng), _orthonormal(9, 5, rng)
        D = O.sign_fix(Zi, Zb)
        got = np.linalg.norm(Zi @ D - Zb)
        brute = min(np.linalg.norm(Zi @ np.diag(s) - Zb) for s in itertools.product([-1.0, 1.0], repeat=5))
        assert got == pytest.approx(brute, abs=1e-13)
        assert set(np.diag(D)) <= {-1.0, 1.0}


def test_k1_sign_fixing_equals_opt():
    """For k = 1 the only orthogonal 1 x 1 matrices are +-1, so OPT and sign-fixing
    coincide (the remark after eq. (4))."""
    _, parts = _small_problem(seed=13)
    Y0 = synth.gaussian_start(12, 1, 14)
    rs = O.localpower(parts, 1, [4, 4, 3], "sign", Y0)
    ro = O.localpower(parts, 1, [4, 4, 3], "opt", Y0)
    assert np.abs(rs["Y"] - ro["Y"]).max() < 1e-13


def test_aggregation_invariances():
    """Sign-fixing and OPT make the aggregate independent of column signs (and, for
    OPT, of any rotation) of the non-base local bases; transforming the base's
    basis transforms the output the same way."""
    rng = _rng(15)
    sizes = [30, 50, 40]          # base = worker 1 (most rows)
    Zl = [_orthonormal(11, 4, rng) for _ in sizes]
    Yl = [rng.standard_normal((11, 4)) for _ in sizes]
    S = np.diag([1.0, -1.0, -1.0, 1.0])
    Q = _orthonormal(4, 4, rng)
    for kind in ("sign", "opt"):
        ref = O.aggregate(Yl, Zl, sizes, kind)
        for i in (0, 2):
            Y2, Z2 = list(Yl), list(Zl)
            Y2[i], Z2[i] = Yl[i] @ S, Zl[i] @ S
            assert np.abs(O.aggregate(Y2, Z2, sizes, kind) - ref).max() < 1e-13
        Y2, Z2 = list(Yl), list(Zl)
        Y2[1], Z2[1] = Yl[1] @ S, Zl[1] @ S
        assert np.abs(O.aggregate(Y2, Z2, sizes, kind) - ref @ S).max() < 1e-13
    ref = O.aggregate(Yl, Zl, sizes, "opt")
    Y2, Z2 = list(Yl), list(Zl)
    Y2[2], Z2[2] = Yl[2] @ Q, Zl[2] @ Q
    assert np.abs(O.aggregate(Y2, Z2, sizes, "opt") - ref).max() < 1e-12
    # vanilla averaging is NOT sign invariant
    Y2, Z2 = list(Yl), list(Zl)
    Y2[0], Z2[0] = Yl[0] @ S, Zl[0] @ S
    assert np.abs(O.aggregate(Y2, Z2, sizes, "identity") - O.aggregate(Yl, Zl, sizes, "identity")).max() > 1e-3


def test_base_is_the_largest_partition_lowest_index_on_ties():
    assert O.base_index([3, 9, 9, 2]) == 1
    assert O.base_index([5, 5, 5]) == 0
    assert O.base_index([1, 2, 3]) == 2


# --------------------------------------------------------------------------- Ritz

def test_ritz_recovers_singular_values():
    """sigma_j = sqrt(n lam_j(Z^T M Z)) equals the singular values of A when Z spans
    the top right singular vectors (LAPACK SVD of A, a different factorisation)."""
    A, parts = _small_problem(seed=16, n=300, sizes=(100, 120, 80))
    _, s, Vt = np.linalg.svd(A, full_matrices=False)
    Zr, sig = O.ritz(parts, O.orth(Vt[:4].T @ _orthonormal(4, 4, _rng(17))))
    assert np.allclose(sig, s[:4], rtol=1e-12)
    for j in range(4):
        assert abs(abs(Zr[:, j] @ Vt[j]) - 1) < 1e-10


def test_rayleigh_quotients_converge_to_top_squared_singular_values():
    A, parts = _small_problem(seed=18, d=8, lam=(8.0, 6.0, 4.0), sigma=0.5, n=900, sizes=(400, 300, 200))
    Y0 = synth.gaussian_start(8, 3, 19)
    r = O.localpower(parts, 3, [4] * 3 + [1] * 80, "sign", Y0)
    _, sig = O.ritz(parts, r["Z"])
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sig ** 2 / A.shape[0], s[:3] ** 2 / A.shape[0], rtol=1e-10)


# --------------------------------------------------------------------------- data model

def test_spiked_model_top_subspace_is_the_spike_basis():
    """For the spiked model the population top-k subspace is U[:, :k]; the sample one
    is within O(sqrt(d/n)/gap) of it (loose check of generator + oracle)."""
    d, lam, sigma, n = 20, np.array([9.0, 6.0, 4.0]), 0.5, 40_000
    A = synth.spiked_rows(n, d, lam, sigma, 21, out_dtype=np.float64, threads=2)
    U = synth.haar_columns(d, 3, 21)
    V, _ = O.top_k_truth([A], 3)
    assert O.subspace_dist(V, U) < 10 * np.sqrt(d / n) * (lam[0] + sigma ** 2) / lam[2]


def test_stored_form_decoders_follow_the_formats():
    # BF16: top half of the FP32 pattern.
    assert O.decode_bf16(np.array([0x3F80, 0xC000, 0x3FC0], dtype=np.uint16)).tolist() == [1.0, -2.0, 1.5]
    # E4M3 (OCP FN): 0x38 = 1, 0x7E = 448 (largest), 0x01 = 2^-9 (smallest subnormal),
    # 0x08 = 2^-6 (smallest normal), 0xB8 = -1, 0x7F = NaN.
    v = O.decode_e4m3(np.array([[0x38, 0x7E, 0x01, 0x08, 0xB8, 0x00]], dtype=np.uint8), np.array([1.0], np.float32))
    assert v.tolist() == [[1.0, 448.0, 2.0 ** -9, 2.0 ** -6, -1.0, 0.0]]
    assert np.isnan(O.decode_e4m3(np.array([[0x7F]], np.uint8), np.array([1.0], np.float32))).all()


def test_encoders_round_to_nearest_within_half_an_ulp():
    rng = _rng(22)
    x = rng.standard_normal((64, 33)).astype(np.float32) * 3
    xb = O.decode_bf16(synth.f32_to_bf16_bits(x))
    assert (np.abs(xb - x) <= 2.0 ** -8 * np.abs(x) + 1e-45).all()
    codes, sc = synth.f32_to_e4m3_rowscaled(x)
    xq = O.decode_e4m3(codes, sc)
    y = x / sc[:, None]
    assert np.abs(y).max() <= 448.0 * (1 + 2 ** -20)
    rel = np.abs(xq - x) / np.maximum(np.abs(x), 2.0 ** -6 * sc[:, None])
    assert rel.max() <= 2.0 ** -4 + 1e-7   # half an ulp of a 3-bit mantissa


# --------------------------------------------------------------------------- residual error rho_t (Def. 3)

def test_residual_error_is_zero_when_all_workers_agree():
    """rho_t = 0 at p_t = 1 (every worker multiplied the broadcast Z) and for
    replicated partitions (identical M_i) at any p."""
    _, parts = _small_problem(seed=21)
    Y0 = _rng(24).standard_normal((12, 3))
    for agg in ("identity", "sign", "opt"):
        out = O.localpower(parts, 3, [1, 1, 1], agg, Y0, keep_trace=True)
        assert max(e["rho"] for e in out["trace"]) < 1e-14
    rep = [parts[0]] * 3
    for agg in ("identity", "sign", "opt"):
        out = O.localpower(rep, 3, [4, 3], agg, Y0, keep_trace=True)
        assert max(e["rho"] for e in out["trace"]) < 1e-12


def test_residual_error_with_opt_matches_the_procrustes_lemma():
    """With OPT, ||Z_i O_i - Z_b||_2 = sqrt(2 - 2 sqrt(1 - dist(Z_i, Z_b)^2)) (App. A),
    a closed form the residual-error routine does not use; and OPT never leaves
    a larger residual than sign-fixing or no alignment on the same bases."""
    rng = _rng(22)
    d, k = 30, 4
    Zb = _orthonormal(d, k, rng)
    Zs = [Zb] + [O.orth(Zb + 0.15 * rng.standard_normal((d, k))) for _ in range(4)]
    sizes = [10, 9, 8, 7, 6]   # worker 0 is the base
    r_opt = O.residual_error(Zs, sizes, "opt")
    want = max(np.sqrt(2 - 2 * np.sqrt(1 - O.subspace_dist(Z, Zb) ** 2)) for Z in Zs[1:])
    assert abs(r_opt - want) < 1e-12
    assert r_opt <= O.residual_error(Zs, sizes, "sign") + 1e-15
    assert r_opt <= O.residual_error(Zs, sizes, "identity") + 1e-15
    # k = 1: sign-fixing is OPT
    Z1 = [Z[:, :1] for Z in Zs]
    assert abs(O.residual_error(Z1, sizes, "sign") - O.residual_error(Z1, sizes, "opt")) < 1e-15


def test_residual_error_is_invariant_to_the_base_basis_sign_flips_of_others():
    """Flipping columns of a non-base basis changes nothing with sign-fixing or OPT."""
    rng = _rng(23)
    Zb = _orthonormal(20, 3, rng)
    Z1 = O.orth(Zb + 0.1 * rng.standard_normal((20, 3)))
    F = np.diag([1.0, -1.0, -1.0])
    for agg in ("sign", "opt"):
        a = O.residual_error([Zb, Z1], [5, 4], agg)
        b = O.residual_error([Zb, Z1 @ F], [5, 4], agg)
        assert abs(a - b) < 1e-12


def test_bf16x2_planes_represent_fp32_within_2_to_minus_17():
    """hi = BF16(a) (the plain encoder), lo = BF16(a - hi); hi + lo is within
    2^-17 |a| of a (and equal to a whenever a has at most 16 significant bits)."""
    rng = _rng(31)
    a = (rng.standard_normal(200_000) * 10.0 ** rng.uniform(-6, 6, 200_000)).astype(np.float32)
    hi, lo = synth.f32_to_bf16x2_planes(a)
    assert np.array_equal(hi, synth.f32_to_bf16_bits(a))
    v = O.decode_bf16(hi) + O.decode_bf16(lo)
    a64 = a.astype(np.float64)
    assert np.all(np.abs(v - a64) <= 2.0 ** -17 * np.abs(a64))
    short = (a.view(np.uint32) & np.uint32(0xFF)) == 0   # 16 significant bits: exact
    assert np.array_equal(v[short], a64[short])


# --------------------------------------------------------------------------- eta (Def. 2)

def _axis_partitions(xs, sizes, d):
    """Partition i holds s_i copies of the row x_i e_i, so M_i = x_i^2 e_i e_i^T."""
    return [np.tile(np.eye(d)[i] * x, (s, 1)) for i, (x, s) in enumerate(zip(xs, sizes))]


def test_eta_closed_form_for_axis_aligned_partitions():
    """With M_i = x_i^2 e_i e_i^T, M = diag(p_j x_j^2) and M_i - M = diag((delta_ij - p_j) x_j^2),
    so ||M_i - M||_2 = max((1 - p_i) x_i^2, max_{j != i} p_j x_j^2) and ||M||_2 = max_j p_j x_j^2.
    Unequal sizes make a 1/n-for-1/s_i or unweighted-mean slip show."""
    cases = [((1.0, 1.0), (5, 5)), ((2.0, 0.5, 1.5), (3, 10, 7)), ((0.3, 3.0, 1.0, 2.0), (40, 1, 9, 20))]
    for xs, sizes in cases:
        q = len(xs)
        parts = _axis_partitions(xs, sizes, q + 2)
        p = np.array(sizes, dtype=np.float64) / sum(sizes)
        x2 = np.array(xs) ** 2
        want = [max((1 - p[i]) * x2[i], max(p[j] * x2[j] for j in range(q) if j != i)) for i in range(q)]
        normM = float(np.max(p * x2))
        e, norms = O.eta(parts)
        np.testing.assert_allclose(norms[:-1], want, rtol=1e-13)
        assert abs(norms[-1] - normM) <= 1e-13 * normM
        assert abs(e - max(want) / normM) <= 1e-13
    assert abs(O.eta(_axis_partitions((1.0, 1.0), (5, 5), 3))[0] - 1.0) < 1e-14


def test_eta_vanishes_without_local_differences_and_is_scale_free():
    """One partition, or identical partitions, give M_i = M (eta = 0); scaling A
    scales every M_i and M alike; more rows per worker shrink eta for iid rows
    (the remark after Def. 2)."""
    _, parts = _small_problem(seed=41)
    assert O.eta(parts[:1])[0] == 0.0
    assert O.eta([parts[0]] * 3)[0] < 1e-14
    e1 = O.eta(parts)[0]
    assert abs(O.eta([2.0 * P for P in parts])[0] - e1) < 1e-12 * e1
    lam = np.array([9.0, 5.0, 3.0, 1.0])
    small = synth.split_rows(synth.spiked_rows(400, 12, lam, 0.3, 44, out_dtype=np.float64, threads=1), [100] * 4)
    big = synth.split_rows(synth.spiked_rows(40_000, 12, lam, 0.3, 44, out_dtype=np.float64, threads=1),
                           [10_000] * 4)
    assert O.eta(big)[0] < 0.3 * O.eta(small)[0]


# --------------------------------------------------------------------------- iteration rank r > k

def test_larger_iteration_rank_nests_the_target_subspace():
    """Alg. 1 takes an iteration rank r >= k.  At p = 1 the iterate spans M^t Y_0,
    so when Y_0's first k columns are the k-column start, span(Z^(k)) lies in
    span(Z^(r)) and dist(Z^(r), U_k) = ||(I - Z^(r) Z^(r)T) U_k||_2 is never the
    larger one; the first k Ritz vectors of the r-column iterate approach U_k
    at least as fast."""
    _, parts = _small_problem(seed=43)
    k, r = 2, 4
    Y0 = _rng(45).standard_normal((12, r))
    V, _ = O.top_k_truth(parts, k)
    last = None
    for T in (1, 3, 6):
        Zk = O.localpower(parts, k, [1] * T, "sign", Y0[:, :k])["Z"]
        Zr = O.localpower(parts, r, [1] * T, "sign", Y0)["Z"]
        assert np.linalg.norm(Zk - Zr @ (Zr.T @ Zk), 2) < 1e-10
        dk, dr = O.subspace_dist(Zk, V), O.subspace_dist(Zr, V)
        assert dr <= dk + 1e-12
        Zr_ritz, _ = O.ritz(parts, Zr)
        assert O.subspace_dist(Zr_ritz[:, :k], V) <= dk + 1e-12
        if last is not None:
            assert dr < last
        last = dr

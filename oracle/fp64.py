"""FP64 CPU oracle for LocalPower (Li, Wang, Chen & Zhang, "Communication-Efficient
Distributed SVD via Local Power Iterations", ICML 2021, arXiv 2002.08014).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark import this module.  The product (the CUDA
library and its Python binding) never imports or calls it, and it shares no
code, header, table or helper with the CUDA path.

Plain, slow, obviously correct: NumPy in FP64, one library routine per step
(matmul, QR, SVD, eigh), no fusion or reordering beyond the paper's own steps.
Each function cites the passage it follows.  Where the paper is silent or
ambiguous the reading taken is stated at the function.

Pins (tests/test_oracle_*.py check each against something other than itself):
  * orth, local step, whole loop at p = 1  -> explicit FP64 subspace iteration
    with M formed densely; ZZ^T = I; diag(R) > 0 convention.
  * m = 1 and replicated partitions        -> subspace iteration with sum(p_t) steps.
  * convergence                            -> brute-force eigh of M (tiny d).
  * procrustes                             -> Lemma (Procrustes identities, App. A),
                                              brute-force minimality over random O.
  * sign_fix                               -> brute force over all 2^k sign matrices.
  * ritz                                   -> singular values of A (LAPACK SVD).
  * subspace_dist                          -> the definition ||UU^T - VV^T||_2 and
                                              principal angles (Def. 1).
  * eta                                    -> closed form for partitions whose rows lie
                                              on distinct coordinate axes; 0 for m = 1 and
                                              replicated partitions; scale invariance.
  * iteration rank r > k                   -> nested subspaces: at p = 1 the r-column
                                              iterate's span contains the k-column one's.
  parity unpinned: the value of the constant-p error floor and the gap between
  OPT and sign-fixing have no closed form (Sec. 4, Thm. 1 gives bounds only);
  they are checked only qualitatively (monotone in p).
"""
from __future__ import annotations

import numpy as np

AGGREGATORS = ("identity", "sign", "opt")


# ---------------------------------------------------------------------------
# Stored forms of A -> exact FP64 values.  These are the oracle's own decoders.
# ---------------------------------------------------------------------------

def decode_bf16(bits: np.ndarray) -> np.ndarray:
    """uint16 BF16 patterns -> FP64 (exact: BF16 is the top half of an FP32)."""
    u = bits.astype(np.uint32) << np.uint32(16)
    return u.view(np.float32).astype(np.float64)


def decode_e4m3(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """uint8 FP8-E4M3 (OCP FN: bias 7, max 448, 0x7F/0xFF = NaN) codes times one
    FP32 scale per row -> FP64 (exact)."""
    c = codes.astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    mant = (c & 7).astype(np.float64)
    mag = np.where(e == 0, mant / 8.0 * 2.0 ** -6, (1.0 + mant / 8.0) * np.exp2(e - 7.0))
    mag = np.where((c & 0x7F) == 0x7F, np.nan, mag)
    return sign * mag * scales.astype(np.float64)[:, None]


def as_f64(part) -> np.ndarray:
    """One partition in any stored form -> its exact FP64 values.

    Accepted forms: an FP32/FP64 array; ("bf16", uint16 bits); ("e4m3", codes, scales).
    """
    if isinstance(part, tuple):
        kind = part[0]
        if kind == "bf16":
            return decode_bf16(part[1])
        if kind == "e4m3":
            return decode_e4m3(part[1], part[2])
        raise ValueError(f"unknown stored form {kind!r}")
    return np.asarray(part, dtype=np.float64)


# ---------------------------------------------------------------------------
# Building blocks
# ---------------------------------------------------------------------------

def weights(sizes) -> np.ndarray:
    """p_i = s_i / n, the fraction of the rows held by worker i (Sec. 2, DPI)."""
    s = np.asarray(sizes, dtype=np.float64)
    return s / s.sum()


def base_index(sizes) -> int:
    """The base worker that every other worker is aligned to: the one holding the
    most rows (Sec. 3, OPT paragraph; the appendix update rule writes argmax p_i).
    Ties go to the lowest index."""
    return int(np.argmax(np.asarray(sizes)))


def orth(Y: np.ndarray) -> np.ndarray:
    """orth(Y): the Q factor of a Householder QR (LAPACK geqrf via numpy), with the
    columns' signs chosen so that diag(R) > 0 (eq. (1); Alg. 1 local computation).
    The paper leaves the sign convention open; diag(R) > 0 is the one a Cholesky-
    based QR produces, and only vanilla averaging depends on it."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def local_step(A_i, Z: np.ndarray) -> np.ndarray:
    """Y_i = M_i Z = (1/s_i) A_i^T (A_i Z) (eq. (2); Alg. 1 local computation)."""
    A = as_f64(A_i)
    return (A.T @ (A @ Z)) / A.shape[0]


def sign_fix(Z_i: np.ndarray, Z_b: np.ndarray) -> np.ndarray:
    """D = diag(sgn<Z_i[:, j], Z_b[:, j]>) (eq. (4)), the minimiser of
    ||Z_i D - Z_b||_F over diagonal +-1 matrices.  sgn(0) is taken as +1."""
    c = np.einsum("dj,dj->j", Z_i, Z_b)
    return np.diag(np.where(c < 0, -1.0, 1.0))


def procrustes(Z_i: np.ndarray, Z_b: np.ndarray) -> np.ndarray:
    """O = W1 W2^T where W1 S W2^T is the SVD of Z_i^T Z_b (eq. (3)): the orthogonal
    k x k matrix minimising ||Z_i O - Z_b||_F."""
    W1, _, W2t = np.linalg.svd(Z_i.T @ Z_b)
    return W1 @ W2t


def align(kind: str, Z_i: np.ndarray, Z_b: np.ndarray) -> np.ndarray:
    """The aligning matrix D in F = {I}, D_k (signs) or O_k (orthogonal) (App. B update rule)."""
    if kind == "identity":
        return np.eye(Z_i.shape[1])
    if kind == "sign":
        return sign_fix(Z_i, Z_b)
    if kind == "opt":
        return procrustes(Z_i, Z_b)
    raise ValueError(f"unknown aggregator {kind!r}")


def aggregate(Y_loc, Z_loc, sizes, kind: str) -> np.ndarray:
    """Y = sum_i p_i Y_i D_i with D_b = I and D_i = align(kind, Z_i, Z_b)
    (Alg. 1 aggregation with eqs. (3)-(4); App. B update rule for Y_t)."""
    w = weights(sizes)
    b = base_index(sizes)
    return sum(w[i] * (Y_loc[i] @ (np.eye(Y_loc[i].shape[1]) if i == b else align(kind, Z_loc[i], Z_loc[b])))
               for i in range(len(Y_loc)))


def residual_error(Z_loc, sizes, kind: str) -> float:
    """rho_t of Def. 3: how far the workers' last local bases are from the base
    worker's, max_i ||Z_i G_i - Z_b||_2 with G_i = I without alignment and the
    Procrustes solution O_i with OPT; with sign-fixing G_i is its diagonal +-1
    matrix (the same form with the aligner the solve uses).  The base worker
    plays the paper's worker 1."""
    b = base_index(sizes)
    worst = 0.0
    for i, Z_i in enumerate(Z_loc):
        if i == b:
            continue
        E = Z_i @ align(kind, Z_i, Z_loc[b]) - Z_loc[b]
        worst = max(worst, float(np.linalg.norm(E, 2)))
    return worst


# ---------------------------------------------------------------------------
# The method
# ---------------------------------------------------------------------------

def localpower(parts, k: int, schedule, agg: str, Y0: np.ndarray, truth: np.ndarray | None = None,
               keep_trace: bool = False) -> dict:
    """LocalPower (Alg. 1 with the aligned aggregation of eqs. (3)-(4) and the
    unified update rule of App. B), counted in rounds.

    parts:    the m row partitions A_i (s_i x d), any form ``as_f64`` accepts.
    schedule: p_t for t = 1..T; round t runs p_t local multiplies and ends with
              one aggregation (one communication; |I_T| = T).
    agg:      "identity" (vanilla), "sign" (eq. (4)) or "opt" (eq. (3)).
    Y0:       the Gaussian start block; Z_0 = orth(Y0).

    Round t (the reading of Alg. 1 used throughout this project):
      1. Z = orth(Y)  -- every worker starts the round from the broadcast Y.
      2. For j = 1..p_t: if j > 1, Z_i = orth(Y_i); then Y_i = M_i Z_i.
      3. D_i = I if p_t = 1 or agg = identity (the remark after eq. (4));
         otherwise D_b = I and D_i aligns the last basis Z_i that worker i
         multiplied to the base worker's Z_b.
      4. Y = sum_i p_i Y_i D_i (Alg. 1 aggregation; App. B eq. for Y_t).
    Output: Z_T = orth(Y) after the last aggregation.
    """
    if agg not in AGGREGATORS:
        raise ValueError(f"unknown aggregator {agg!r}")
    As = [as_f64(P) for P in parts]
    sizes = [A.shape[0] for A in As]
    b = base_index(sizes)
    m = len(As)
    Y = np.asarray(Y0, dtype=np.float64)
    trace = []
    for p_t in schedule:
        Z = orth(Y)
        Z_loc = [Z] * m
        Y_loc = [None] * m
        for j in range(int(p_t)):
            for i in range(m):
                if j > 0:
                    Z_loc[i] = orth(Y_loc[i])
                Y_loc[i] = local_step(As[i], Z_loc[i])
        Y = aggregate(Y_loc, Z_loc, sizes, "identity" if int(p_t) == 1 else agg)
        if keep_trace or truth is not None:
            entry = {"p": int(p_t)}
            if keep_trace:
                entry["Z"] = orth(Y)
                entry["rho"] = residual_error(Z_loc, sizes, agg)
            if truth is not None:
                entry["dist"] = subspace_dist(orth(Y), truth)
            trace.append(entry)
    return {"Z": orth(Y), "Y": Y, "trace": trace, "rounds": len(schedule),
            "local_steps": int(sum(int(p) for p in schedule)), "base": b}


def ritz(parts, Z: np.ndarray):
    """Rayleigh-Ritz on span(Z) (a final step added to the method; the paper stops
    at orth(Y)): H = Z^T M Z with M = (1/n) sum_i A_i^T A_i, H = W diag(lam) W^T
    with lam descending; returns (Z W, sigma) with sigma_j = sqrt(n lam_j), the
    estimates of the top singular values of A."""
    As = [as_f64(P) for P in parts]
    n = sum(A.shape[0] for A in As)
    MZ = sum(A.T @ (A @ Z) for A in As) / n
    H = Z.T @ MZ
    H = 0.5 * (H + H.T)
    lam, W = np.linalg.eigh(H)
    order = np.argsort(lam)[::-1]
    lam, W = lam[order], W[:, order]
    return Z @ W, np.sqrt(np.maximum(lam, 0.0) * n)


# ---------------------------------------------------------------------------
# Metrics and brute-force references
# ---------------------------------------------------------------------------

def subspace_dist(U: np.ndarray, V: np.ndarray) -> float:
    """dist(U, V) = ||U U^T - V V^T||_2 = sin theta_k (Def. 1 and the equivalent
    forms in App. A), evaluated as ||(I - U U^T) V||_2 after re-orthonormalising
    both bases in FP64; this form keeps full relative accuracy for tiny angles."""
    Uo, Vo = orth(U), orth(V)
    R = Vo - Uo @ (Uo.T @ Vo)
    return float(np.linalg.norm(R, 2))


def principal_cosines(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """cos theta_l = sigma_l(U^T V), descending (Sec. 4, after Def. 1)."""
    return np.linalg.svd(orth(U).T @ orth(V), compute_uv=False)


def explicit_M(parts) -> np.ndarray:
    """M = (1/n) sum_i A_i^T A_i formed densely (Def. 2)."""
    As = [as_f64(P) for P in parts]
    n = sum(A.shape[0] for A in As)
    return sum(A.T @ A for A in As) / n


def top_k_truth(parts, k: int):
    """Top-k eigenvectors / eigenvalues of M by a full symmetric eigendecomposition."""
    M = explicit_M(parts)
    lam, V = np.linalg.eigh(M)
    return V[:, ::-1][:, :k], lam[::-1]


def eta(parts):
    """eta = max_i ||M_i - M||_2 / ||M||_2 with M_i = (1/s_i) A_i^T A_i and
    M = sum_i p_i M_i (Def. 2), each spectral norm from a full symmetric
    eigendecomposition.  Returns (eta, [||M_i - M||_2 ...] + [||M||_2])."""
    As = [as_f64(P) for P in parts]
    sizes = [A.shape[0] for A in As]
    p = weights(sizes)
    Ms = [A.T @ A / A.shape[0] for A in As]
    M = sum(pi * Mi for pi, Mi in zip(p, Ms))
    norms = [float(np.max(np.abs(np.linalg.eigvalsh(Mi - M)))) for Mi in Ms]
    normM = float(np.max(np.abs(np.linalg.eigvalsh(M))))
    return max(norms) / normM, np.array(norms + [normM])


def subspace_iteration(M: np.ndarray, Y0: np.ndarray, steps: int) -> np.ndarray:
    """Plain power/subspace iteration Z <- orth(M Z) (eq. (1)) from Z = orth(Y0)."""
    Z = orth(Y0)
    for _ in range(steps):
        Z = orth(M @ Z)
    return Z

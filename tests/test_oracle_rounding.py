"""Pins of the oracle's rounding algorithms (Algorithms 1-7 and the Section 3.2
truncation) against brute force on full tensors, closed forms and invariants."""
import numpy as np
import pytest

import oracle as O
import synth
from tests._tt_helpers import (unfold, orth, tt_svd_full, rel, left_part_bruteforce,
                               right_part_bruteforce, full_from_cores_bruteforce)


def _tt(seed, dims, ranks):
    return synth.gaussian_tt(synth.rng_for(seed, 11), dims, ranks)


def _const(N, r):
    return [1] + [r] * (N - 1) + [1]


# ---------------------------------------------------------------- Algorithm 3

def test_partial_contractions_rl_definition():
    """W_n = H(X_{n+1:N}) H(Y_{n+1:N})^T (Section 2.3), by brute force."""
    dims = [3, 2, 3, 2]
    X = _tt(1, dims, [1, 2, 3, 2, 1])
    Y = _tt(2, dims, [1, 3, 2, 4, 1])
    W = O.partial_contractions_rl(X, Y)
    for n in range(1, 4):
        ref = right_part_bruteforce(X, n) @ right_part_bruteforce(Y, n).T
        np.testing.assert_allclose(W[n], ref, rtol=1e-12, atol=1e-15)


def test_partial_contractions_lr_definition():
    dims = [3, 2, 3, 2]
    Y = _tt(3, dims, [1, 2, 3, 2, 1])
    L = _tt(4, dims, [1, 3, 2, 4, 1])
    WL = O.partial_contractions_lr(Y, L)
    for n in range(1, 4):
        ref = left_part_bruteforce(L, n).T @ left_part_bruteforce(Y, n)
        np.testing.assert_allclose(WL[n], ref, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------- Algorithms 1 and 2

def test_orthogonalize_rl_and_lr():
    dims = [3, 4, 2, 3]
    Y = _tt(5, dims, [1, 3, 4, 3, 1])
    F = full_from_cores_bruteforce(Y)
    X = O.orthogonalize_rl(Y)
    assert rel(O.full(X), F) < 1e-13
    for n in range(1, 4):
        Hn = O.H(X[n])
        np.testing.assert_allclose(Hn @ Hn.T, np.eye(Hn.shape[0]), atol=1e-14)
    Xl = O.orthogonalize_lr(Y)
    assert rel(O.full(Xl), F) < 1e-13
    for n in range(3):
        Vn = O.V(Xl[n])
        np.testing.assert_allclose(Vn.T @ Vn, np.eye(Vn.shape[1]), atol=1e-14)


def test_det_rounding_singular_values_are_those_of_the_unfoldings():
    """Algorithm 2 with eps0 = 0: the singular values of R at step n are the
    singular values of the unfolding Y_(1:n) (up to the rank)."""
    dims = [3, 4, 3, 2]
    Y = _tt(6, dims, [1, 3, 4, 2, 1])
    F = full_from_cores_bruteforce(Y)
    X, svs = O.tt_round_det(Y, 0.0, return_sv=True)
    for n in range(1, 4):
        s_ref = np.linalg.svd(unfold(F, n), compute_uv=False)
        k = len(svs[n - 1])
        np.testing.assert_allclose(svs[n - 1], s_ref[:k], rtol=1e-10, atol=1e-14 * s_ref[0])
        assert np.all(s_ref[k:] <= 1e-12 * s_ref[0])
    assert rel(O.full(X), F) < 1e-12


@pytest.mark.parametrize("eps0", [1e-1, 1e-2, 1e-4])
def test_det_rounding_error_bound(eps0):
    """||X - Y|| <= eps0 ||Y|| (Algorithm 2 guarantee)."""
    dims = [4, 3, 4, 3, 4]
    Y = O.block_sum([_tt(7, dims, _const(5, 3)), synth.scale_tt(_tt(8, dims, _const(5, 4)), 0.05)])
    X = O.tt_round_det(Y, eps0)
    F = full_from_cores_bruteforce(Y)
    err = np.linalg.norm(O.full(X) - F)
    assert err <= eps0 * np.linalg.norm(F) * (1 + 1e-10)
    if eps0 >= 1e-2:   # the 0.05-weighted summand falls below the threshold
        assert sum(O.ranks_of(X)) < sum(O.ranks_of(Y))


def test_det_rounding_equals_tt_svd_of_full_tensor():
    dims = [3, 4, 3, 4]
    Y = _tt(9, dims, [1, 3, 5, 3, 1])
    F = full_from_cores_bruteforce(Y)
    X = O.tt_round_det(Y, 0.0, max_rank=2)
    ref = tt_svd_full(F, [1, 2, 2, 2, 1])
    assert rel(O.full(X), O.full(ref)) < 1e-10


def test_truncate_left_orthogonal_matches_rl_tt_svd():
    """Section 3.2 truncation (right-to-left sweep on a left-orthogonal TT):
    singular values are those of the unfoldings and fixed-rank output equals the
    right-to-left TT-SVD of the full tensor."""
    dims = [3, 4, 3, 4]
    Y = O.orthogonalize_lr(_tt(10, dims, [1, 3, 5, 3, 1]))
    F = full_from_cores_bruteforce(Y)
    X, svs = O.truncate_left_orthogonal(Y, 0.0, return_sv=True)
    for n in range(1, 4):
        s_ref = np.linalg.svd(unfold(F, n), compute_uv=False)
        k = len(svs[n])
        np.testing.assert_allclose(svs[n], s_ref[:k], rtol=1e-10, atol=1e-14 * s_ref[0])
    X2 = O.truncate_left_orthogonal(Y, 0.0, max_rank=2)
    # right-to-left TT-SVD = left-to-right TT-SVD of the mode-reversed tensor
    ref = tt_svd_full(F.transpose(3, 2, 1, 0).copy(), [1, 2, 2, 2, 1])
    assert rel(O.full(X2), O.full(ref).transpose(3, 2, 1, 0)) < 1e-10
    for n in range(1, 4):   # output is right-orthogonal
        Hn = O.H(X2[n])
        np.testing.assert_allclose(Hn @ Hn.T, np.eye(Hn.shape[0]), atol=1e-13)


@pytest.mark.parametrize("eps0", [1e-2, 1e-5])
def test_truncate_left_orthogonal_error_bound(eps0):
    dims = [4, 3, 4, 3, 4]
    Y = O.block_sum([_tt(11, dims, _const(5, 3)), synth.scale_tt(_tt(12, dims, _const(5, 4)), 1e-3)])
    Xl = O.orthogonalize_lr(Y)
    X = O.truncate_left_orthogonal(Xl, eps0)
    F = full_from_cores_bruteforce(Y)
    assert np.linalg.norm(O.full(X) - F) <= eps0 * np.linalg.norm(F) * (1 + 1e-10)


# ----------------------------------------------------------- Algorithms 5, 7

def _projection_reference(F, omegas_full):
    """X_hat_(1:N-1) = Pi_{N-1} F_(1:N-1), Pi_n the orthogonal projector onto
    range((Pi_{n-1} (x) I) F_(1:n) Omega_n) (the randomized range finder of
    Section 2.2 applied bond by bond)."""
    dims = F.shape
    N = len(dims)
    Pi = np.ones((1, 1))
    for n in range(1, N):
        A = np.kron(Pi, np.eye(dims[n - 1])) @ unfold(F, n) @ omegas_full[n]
        Qn = orth(A)
        Pi = Qn @ Qn.T
    return (Pi @ unfold(F, N - 1)).reshape(dims)


def test_randorth_equals_bond_by_bond_projection():
    dims = [3, 4, 3, 4, 3]
    Y = _tt(13, dims, [1, 3, 6, 6, 3, 1])
    ell = [1, 2, 3, 3, 2, 1]
    R = _tt(14, dims, ell)
    X = O.round_randorth(Y, R)
    assert O.ranks_of(X) == ell
    F = full_from_cores_bruteforce(Y)
    om = [None] + [right_part_bruteforce(R, n).T for n in range(1, 5)]
    ref = _projection_reference(F, om)
    assert rel(O.full(X), ref) < 1e-10
    # left-orthogonal output and Pythagoras (single orthogonal projection)
    for n in range(4):
        Vn = O.V(X[n])
        np.testing.assert_allclose(Vn.T @ Vn, np.eye(Vn.shape[1]), atol=1e-13)
    FX = O.full(X)
    assert abs(np.linalg.norm(F) ** 2 - np.linalg.norm(FX) ** 2 - np.linalg.norm(F - FX) ** 2) < 1e-10 * np.linalg.norm(F) ** 2


def test_randorth_exact_recovery():
    """Target ranks >= the true TT-ranks: the rounding reproduces the tensor."""
    dims = [5, 6, 5, 6, 5, 6]
    Y = _tt(15, dims, _const(6, 3))
    Ysum = O.block_sum([Y, Y])                         # X + X, formal rank 6
    R = _tt(16, dims, _const(6, 4))
    X = O.round_randorth(Ysum, R)
    assert O.diff_norm(X, O.block_sum([Y], [2.0])) <= 1e-12 * O.norm(Ysum)
    Xt = O.truncate_left_orthogonal(X, 1e-10)
    assert O.ranks_of(Xt) == _const(6, 3)


def test_randorth_invariances():
    """Output depends only on the represented tensor and the sketch: gauge
    transforms of Y and scaling of sketch cores leave it unchanged;
    round(cY) = c round(Y)."""
    dims = [4, 5, 4, 5]
    Y = _tt(17, dims, [1, 4, 5, 4, 1])
    R = _tt(18, dims, [1, 2, 3, 2, 1])
    X = O.round_randorth(Y, R)
    Yg = synth.gauge_scramble(synth.rng_for(19), Y)
    assert O.diff_norm(O.round_randorth(Yg, R), X) <= 1e-11 * O.norm(X)
    Rs = [c * s for c, s in zip(R, [3.0, 0.25, 7.0, 0.5])]
    assert O.diff_norm(O.round_randorth(Y, Rs), X) <= 1e-11 * O.norm(X)
    Xc = O.round_randorth(synth.scale_tt(Y, -2.5), R)
    assert O.diff_norm(Xc, synth.scale_tt(X, -2.5)) <= 1e-11 * O.norm(Xc)


def test_sum_randorth_equals_randorth_of_formed_sum():
    """Algorithm 7 == Algorithm 5 applied to the block TT-sum with the same
    sketch (derivation of Section 3.4)."""
    dims = [3, 4, 3, 4, 3]
    Ys = [_tt(20 + j, dims, [1, r, r + 1, r + 1, r, 1]) for j, r in enumerate([2, 3, 1, 2])]
    R = _tt(30, dims, [1, 3, 4, 4, 3, 1])
    coeffs = [1.0, -0.5, 2.0, 0.75]
    X7 = O.round_sum_randorth(Ys, R, coeffs)
    X5 = O.round_randorth(O.block_sum(Ys, coeffs), R)
    assert O.diff_norm(X7, X5) <= 1e-13 * O.norm(X5)
    # permuting summands does not change the represented output
    perm = [2, 0, 3, 1]
    Xp = O.round_sum_randorth([Ys[p] for p in perm], R, [coeffs[p] for p in perm])
    assert O.diff_norm(Xp, X7) <= 1e-12 * O.norm(X7)
    # and it is the bond-by-bond projection of the full sum
    F = sum(c * full_from_cores_bruteforce(Y) for c, Y in zip(coeffs, Ys))
    om = [None] + [right_part_bruteforce(R, n).T for n in range(1, 5)]
    assert rel(O.full(X7), _projection_reference(F, om)) < 1e-10


def test_sum_randorth_x_plus_x_recovers_rank():
    dims = [6] * 6
    Y = _tt(31, dims, _const(6, 3))
    R = _tt(32, dims, _const(6, 5))
    X = O.round_sum_randorth([Y, Y], R)
    assert O.diff_norm(X, synth.scale_tt(Y, 2.0)) <= 1e-12 * 2 * O.norm(Y)
    assert O.ranks_of(O.truncate_left_orthogonal(X, 1e-9)) == _const(6, 3)


# ------------------------------------------------------------- Algorithm 4

def test_orthrand_equals_projection_and_recovers():
    dims = [3, 4, 3, 4, 3]
    Y = _tt(33, dims, [1, 3, 6, 6, 3, 1])
    ell = [1, 2, 3, 3, 2, 1]
    Yo = O.orthogonalize_rl(Y)
    rng = synth.rng_for(34)
    Om = [None] + [synth.gaussian_matrix(rng, O.ranks_of(Yo)[n], ell[n]) for n in range(1, 5)]
    X = O.round_orthrand(Y, Om)
    F = full_from_cores_bruteforce(Y)
    om = [None] + [right_part_bruteforce(Yo, n).T @ Om[n] for n in range(1, 5)]
    assert rel(O.full(X), _projection_reference(F, om)) < 1e-10
    # exact recovery
    Y3 = _tt(35, [5] * 5, _const(5, 3))
    Om3 = [None] + [synth.gaussian_matrix(rng, 3, 4) for _ in range(4)]
    assert O.diff_norm(O.round_orthrand(Y3, Om3), Y3) <= 1e-12 * O.norm(Y3)


# ------------------------------------------------------------- Algorithm 6

def test_twosided_matrix_case_is_generalized_nystrom():
    """N = 2: X_hat = (Y Omega)(Psi Y Omega)^+(Psi Y) (Eq. of Section 2.2)."""
    rng = synth.rng_for(36)
    Y = _tt(37, [12, 10], [1, 6, 1])
    L = _tt(38, [12, 10], [1, 3, 1])
    Rk = _tt(39, [12, 10], [1, 5, 1])
    X = O.round_twosided(Y, L, Rk)
    A = O.full(Y)
    Psi = L[0][0].T               # l x I_1
    Om = Rk[1][:, :, 0].T         # I_2 x rho
    ref = (A @ Om) @ np.linalg.pinv(Psi @ A @ Om) @ (Psi @ A)
    assert rel(O.full(X), ref) < 1e-11


def test_twosided_equals_bondwise_nystrom_and_recovers():
    dims = [3, 4, 3, 4]
    Y = _tt(40, dims, [1, 3, 5, 3, 1])
    ell = [1, 2, 3, 2, 1]
    rho = [1, 3, 5, 3, 1]
    L = _tt(41, dims, ell)
    Rk = _tt(42, dims, rho)
    X = O.round_twosided(Y, L, Rk)
    # brute force: insert P_n = W^R_n (W^L_n W^R_n)^+ W^L_n on every bond
    cores = [c.copy() for c in Y]
    for n in range(1, 4):
        WL = left_part_bruteforce(L, n).T @ left_part_bruteforce(Y, n)
        WR = right_part_bruteforce(Y, n) @ right_part_bruteforce(Rk, n).T
        P = WR @ np.linalg.pinv(WL @ WR) @ WL
        cores[n - 1] = np.einsum("aib,bc->aic", cores[n - 1], P)
    assert rel(O.full(X), full_from_cores_bruteforce(cores)) < 1e-9
    # exact recovery when rank <= l <= rho
    Y2 = _tt(43, [5] * 5, _const(5, 3))
    X2 = O.round_twosided(Y2, _tt(44, [5] * 5, _const(5, 4)), _tt(45, [5] * 5, _const(5, 6)))
    assert O.diff_norm(X2, Y2) <= 1e-10 * O.norm(Y2)


def test_twosided_orth_same_tensor_left_orthogonal_and_truncation_bound():
    """The orthogonalizing restructure of Algorithm 6 (Section 3.3, reading in
    round_sum_twosided_orth): the same full tensor as Algorithm 6 built by brute
    force from the bond-wise Nystrom projectors, left-orthogonal cores, and with
    a tolerance the Section 3.2 bound ||X_out - X|| <= tol ||X||."""
    dims = [3, 4, 3, 4]
    Ys = [_tt(46, dims, [1, 2, 3, 2, 1]), _tt(47, dims, [1, 3, 2, 2, 1])]
    coeffs = [0.7, -1.3]
    ell = [1, 3, 4, 3, 1]
    rho = [1, 4, 5, 4, 1]
    L, Rk = _tt(48, dims, ell), _tt(49, dims, rho)
    Ysum = O.block_sum(Ys, coeffs)
    cores = [c.copy() for c in Ysum]
    for n in range(1, 4):
        WL = left_part_bruteforce(L, n).T @ left_part_bruteforce(Ysum, n)
        WR = right_part_bruteforce(Ysum, n) @ right_part_bruteforce(Rk, n).T
        P = WR @ np.linalg.pinv(WL @ WR) @ WL
        cores[n - 1] = np.einsum("aib,bc->aic", cores[n - 1], P)
    ref = full_from_cores_bruteforce(cores)
    X = O.round_sum_twosided_orth(Ys, L, Rk, coeffs)
    assert rel(O.full(X), ref) < 1e-9
    for n in range(3):
        Vn = O.V(X[n])
        assert np.abs(Vn.T @ Vn - np.eye(Vn.shape[1])).max() < 1e-13
    for tol in (2e-1, 9e-1):
        Xt = O.round_sum_twosided_orth(Ys, L, Rk, coeffs, eps0=tol)
        assert O.diff_norm(Xt, X) <= tol * O.norm(X) * (1 + 1e-12)
    assert sum(O.ranks_of(Xt)) < sum(O.ranks_of(X))


def test_twosided_orth_recovers_low_rank_sum():
    """X + X of rank r <= l <= rho: the restructured Two-Sided result with a
    tolerance is 2X at rank r (generalized Nystrom identity, Section 3.3)."""
    dims = [5] * 5
    Y = _tt(51, dims, _const(5, 3))
    X = O.round_sum_twosided_orth([Y, Y], _tt(52, dims, _const(5, 4)), _tt(53, dims, _const(5, 6)), eps0=1e-10)
    assert O.ranks_of(X) == _const(5, 3)
    assert O.diff_norm(X, synth.scale_tt(Y, 2.0)) <= 1e-10 * O.norm(Y)


# ------------------------------------------------- Section 4.1 / Appendix C

def test_accuracy_ordering_perturbed_tt():
    """Section 4.1 (qualitative): deterministic rounding is the most accurate,
    and the randomized errors shrink as the perturbation shrinks."""
    dims = [6] * 6
    errs = {}
    for eps in (1e-2, 1e-6):
        acc = {"det": [], "rto": [], "otr": [], "2sr": []}
        for seed in range(3):
            Y = O.block_sum([_tt(50 + seed, dims, _const(6, 4)),
                             synth.scale_tt(_tt(60 + seed, dims, _const(6, 4)), eps)])
            F = O.norm(Y)
            l = 5
            acc["det"].append(O.diff_norm(O.tt_round_det(Y, 0.0, max_rank=l), Y) / F)
            R = _tt(70 + seed, dims, _const(6, l))
            acc["rto"].append(O.diff_norm(O.round_randorth(Y, R), Y) / F)
            rng = synth.rng_for(80 + seed)
            ro = O.ranks_of(O.orthogonalize_rl(Y))
            Om = [None] + [synth.gaussian_matrix(rng, ro[n], l) for n in range(1, 6)]
            acc["otr"].append(O.diff_norm(O.round_orthrand(Y, Om), Y) / F)
            Rr = _tt(90 + seed, dims, _const(6, int(np.ceil(1.5 * l))))
            acc["2sr"].append(O.diff_norm(O.round_twosided(Y, R, Rr), Y) / F)
        errs[eps] = {k: float(np.mean(v)) for k, v in acc.items()}
        assert errs[eps]["det"] <= min(errs[eps]["rto"], errs[eps]["otr"], errs[eps]["2sr"]) * (1 + 1e-8)
    for k in ("rto", "otr", "2sr"):
        assert errs[1e-6][k] < errs[1e-2][k]


def test_hilbert_tt_randomized_matches_deterministic():
    """Appendix C (scaled down): on a Hilbert-type TT with fast spectral decay,
    Randomize-then-Orthogonalize is about as accurate as TT-SVD rounding."""
    dims = [6, 8, 10, 12, 14]
    Y = synth.hilbert_tt(dims, [1, 4, 5, 6, 7, 1])
    F = O.norm(Y)
    for r in (2, 3):
        e_det = O.diff_norm(O.tt_round_det(Y, 0.0, max_rank=r), Y) / F
        R = _tt(100 + r, dims, O.clamp_ranks(dims, _const(5, r + 2)))
        Xr = O.truncate_left_orthogonal(O.round_randorth(Y, R), 0.0, max_rank=r)
        e_rto = O.diff_norm(Xr, Y) / F
        assert e_rto < 10 * e_det and e_det < 10 * e_rto


def test_clamp_ranks():
    assert O.clamp_ranks([2, 3, 100, 2], [1, 50, 50, 50, 1]) == [1, 2, 6, 2, 1]


def test_qr_pos_is_the_unique_positive_diagonal_qr():
    """For full column rank, R of the positive-diagonal thin QR is the
    transposed Cholesky factor of A^T A (uniqueness of that factorization)."""
    from oracle.rounding import qr_pos
    A = synth.rng_for(120).standard_normal((40, 7))
    Q, R = qr_pos(A)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(R, np.linalg.cholesky(A.T @ A).T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)

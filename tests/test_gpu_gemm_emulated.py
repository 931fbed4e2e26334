"""The emulated FP64 product of the mixed path (tt_gemm_emulated_f64) against
the plain definition of a matrix product: exact results where the digits hold
the inputs exactly, the stated error bound on random inputs (reference in
extended precision), scale invariance, determinism, strided views, ragged and
degenerate shapes."""
import numpy as np
import pytest
import torch

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu


def _run(A, B, s, C=None, alpha=1.0, beta=0.0):
    Cd = None if C is None else torch.from_numpy(C).cuda()
    out = tt.tt_gemm_emulated_f64(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=alpha, beta=beta,
                                  digits=s)
    torch.cuda.synchronize()
    return out.cpu().numpy()


SHAPES = [(200, 30, 3000), (3000, 30, 200), (30, 200, 3000), (1, 1, 1), (129, 33, 65), (1000, 30, 10),
          (7, 300, 64), (256, 64, 129), (30, 30, 3000)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("s", [5, 8])
def test_integer_inputs_exact(M, N, K, s):
    # |entries| < 2^20 fill three 7-bit digits (relative to 2^{e+2}, e <= 19),
    # so every nonzero digit pair has level <= 6 and is kept for s >= 5; the
    # product sums stay below 2^53, so the result must equal the exact product.
    rng = np.random.default_rng(M * 1009 + N * 31 + K + s)
    A = rng.integers(-(1 << 20) + 1, 1 << 20, size=(M, K)).astype(np.float64)
    B = rng.integers(-(1 << 20) + 1, 1 << 20, size=(K, N)).astype(np.float64)
    C = _run(A, B, s)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("s", [1, 2, 3])
def test_small_integers_exact_with_few_digits(s):
    rng = np.random.default_rng(s)
    A = rng.integers(-63, 64, size=(150, 70)).astype(np.float64)
    B = rng.integers(-63, 64, size=(70, 40)).astype(np.float64)
    assert np.array_equal(_run(A, B, s), A @ B)


def _exact(A, B):
    return (A.astype(np.longdouble) @ B.astype(np.longdouble))


@pytest.mark.parametrize("M,N,K", [(200, 30, 1500), (600, 30, 200), (30, 100, 700), (129, 33, 65)])
@pytest.mark.parametrize("s", [2, 5, 8])
def test_random_error_bound(M, N, K, s):
    rng = np.random.default_rng(M + N + K + 100 * s)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, size=(1, N)))
    C = _run(A, B, s).astype(np.longdouble)
    ref = _exact(A, B)
    scale = np.abs(A).max(axis=1, keepdims=True) * np.abs(B).max(axis=0, keepdims=True)
    bound = K * 2.0 ** (4 - 7 * s) * scale + 2.0 ** -52 * np.abs(ref)
    err = np.abs(C - ref)
    assert np.all(err <= bound)
    if s == 8:
        # FP64 class: typical error at the rounding level of the result
        rel = np.abs(C - ref) / np.maximum(np.abs(ref), 1e-300)
        assert float(np.median(rel)) < 1e-15


def test_scale_invariance_bitwise():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((300, 500))
    B = rng.standard_normal((500, 30))
    C = _run(A, B, 8)
    C2 = _run(A * 2.0 ** 300, B * 2.0 ** -500, 8)
    assert np.array_equal(C2, C * 2.0 ** -200)


def test_deterministic_bitwise():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((200, 3000))
    B = rng.standard_normal((3000, 30))
    assert np.array_equal(_run(A, B, 8), _run(A, B, 8))


def test_wide_dynamic_range_rows():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((130, 300))
    A[0] *= 1e250
    A[1] *= 1e-250
    A[2, ::3] *= 1e-30
    B = rng.standard_normal((300, 20))
    C = _run(A, B, 8).astype(np.longdouble)
    ref = _exact(A, B)
    scale = np.abs(A).max(axis=1, keepdims=True) * np.abs(B).max(axis=0, keepdims=True)
    assert np.all(np.abs(C - ref) <= 300 * 2.0 ** (4 - 56) * scale + 2.0 ** -52 * np.abs(ref))


def test_strided_views_and_alpha_beta():
    rng = np.random.default_rng(8)
    At = rng.standard_normal((400, 150))       # A = At^T: rows contiguous along M
    Bw = rng.standard_normal((400, 90))        # B = Bw[:, ::3]: column stride 3
    A = torch.from_numpy(At).cuda().t()
    B = torch.from_numpy(Bw).cuda()[:, ::3]
    C0 = rng.standard_normal((30, 150))
    Cd = torch.from_numpy(C0.copy()).cuda().t()  # C is a transposed view
    tt.tt_gemm_emulated_f64(A, B, Cd, alpha=0.5, beta=-2.0, digits=8)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy()
    ref = 0.5 * (At.T @ Bw[:, ::3]) - 2.0 * C0.T
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_zero_and_degenerate():
    A = np.zeros((140, 70))
    B = np.random.default_rng(9).standard_normal((70, 33))
    assert np.array_equal(_run(A, B, 8), np.zeros((140, 33)))
    # K = 0: C = beta C
    A0 = np.zeros((5, 0))
    B0 = np.zeros((0, 4))
    C0 = np.arange(20.0).reshape(5, 4)
    assert np.array_equal(_run(A0, B0, 8, C=C0.copy(), beta=3.0), 3.0 * C0)
    # a zero column of B and a zero row of A
    rng = np.random.default_rng(10)
    A = rng.standard_normal((64, 100))
    B = rng.standard_normal((100, 8))
    A[3] = 0.0
    B[:, 5] = 0.0
    C = _run(A, B, 8)
    assert np.all(C[3] == 0.0) and np.all(C[:, 5] == 0.0)


def test_invalid_arguments_rejected():
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTError):
        tt.tt_gemm_emulated_f64(A, A, digits=0)
    with pytest.raises(tt.TTError):
        tt.tt_gemm_emulated_f64(A, A, digits=9)


def test_nonfinite_rows_and_columns_give_nan():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((140, 70))
    B = rng.standard_normal((70, 20))
    A[5, 3] = np.nan
    A[7, 0] = np.inf
    B[2, 4] = -np.inf
    C = _run(A, B, 8)
    assert np.all(np.isnan(C[5])) and np.all(np.isnan(C[7])) and np.all(np.isnan(C[:, 4]))
    keep_r = [r for r in range(140) if r not in (5, 7)]
    keep_c = [c for c in range(20) if c != 4]
    A2, B2 = A[keep_r], B[:, keep_c]
    assert np.allclose(C[np.ix_(keep_r, keep_c)], A2 @ B2, rtol=1e-13, atol=1e-13)


@pytest.fixture
def _gemm_mode_restore():
    yield
    tt.set_gemm_mode(tt.GEMM_AUTO)


@pytest.mark.parametrize("M,N,K,digits", [(300, 30, 200, 8), (30, 200, 3000, 8), (2048, 24, 480, 6),
                                          (130, 70, 1100, 2), (5, 3, 7, 4), (257, 33, 64, 8)])
def test_fused_and_three_pass_products_are_bit_identical(M, N, K, digits, _gemm_mode_restore):
    """The single-launch product (exponent scan and digit split in the product
    kernel) and the three-pass form compute the same integers: equal bits."""
    rng = np.random.default_rng(M + 7 * N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, size=(1, N)))
    A[M // 2, :] = 0.0
    C0 = rng.standard_normal((M, N))
    outs = []
    for mode in (tt.GEMM_THREE_PASS, tt.GEMM_FUSED):
        tt.set_gemm_mode(mode)
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        Cd = torch.from_numpy(C0.copy()).cuda()
        tt.tt_gemm_emulated_f64(Ad, Bd, Cd, alpha=-0.5, beta=1.0, digits=digits)
        Ct = torch.from_numpy(C0.T.copy()).cuda().t()      # a transposed output view, A given transposed
        tt.tt_gemm_emulated_f64(torch.from_numpy(A.T.copy()).cuda().t(), Bd, Ct, digits=digits)
        torch.cuda.synchronize()
        outs.append((Cd.cpu(), Ct.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    ref = A @ B
    scale = np.abs(A).max(axis=1, keepdims=True) * np.abs(B).max(axis=0, keepdims=True)
    assert np.all(np.abs(outs[1][1].numpy() - ref) <= K * 2.0 ** (4 - 7 * digits) * scale + 2.0 ** -52 * np.abs(ref))


def test_fused_products_flag_non_finite_rows(_gemm_mode_restore):
    tt.set_gemm_mode(tt.GEMM_FUSED)
    A = np.ones((40, 50))
    A[3, 7] = np.inf
    B = np.ones((50, 20))
    B[9, 5] = np.nan
    C = _run(A, B, 8)
    assert np.all(np.isnan(C[3, :])) and np.all(np.isnan(C[:, 5]))
    mask = np.ones_like(C, dtype=bool)
    mask[3, :] = False
    mask[:, 5] = False
    assert np.all(C[mask] == 50.0)


@pytest.mark.parametrize("tol", [0.0, 1e-8])
def test_mixed_rounding_identical_in_both_gemm_modes(tol, _gemm_mode_restore):
    import synth
    dims = [30, 40, 36, 30, 40]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(650, j), dims, [1] + [r] * (N - 1) + [1]) for j, r in enumerate([4, 6, 5])]
    ell = [1] + [12] * (N - 1) + [1]
    Yd = [[torch.from_numpy(c).cuda() for c in Y] for Y in Ys]
    res = []
    for mode in (tt.GEMM_THREE_PASS, tt.GEMM_FUSED):
        tt.set_gemm_mode(mode)
        res.append([c.cpu() for c in tt.tt_round_sum_rand(Yd, ell, seed=3, tol=tol, precision="mixed")])
    for a, b in zip(*res):
        assert torch.equal(a, b)

"""Mixed-precision sum rounding (tensor-core split FP64 contractions) against
the FP64 GPU path and the oracle; the accuracy gate of the mixed path is its
rounding error relative to the oracle's (<= 1.1x) on the same sketch."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu


def test_tcgen05_fp32_accumulation_exact_up_to_2_24():
    """The digit products rely on exact fp32 accumulation of integer sums below
    2^24: K = 1024 products of 127 * 127 sum to 16,516,096 < 2^24."""
    from paper_2110_04393_gb300 import _native
    lib = _native.lib()
    M, N, K = 128, 16, 1024
    a = np.full((M, K), 127.0)
    b = np.full((N, K), 127.0)
    b[1::2] = -127.0
    A = torch.from_numpy(a).to("cuda", torch.bfloat16).contiguous()
    B = torch.from_numpy(b).to("cuda", torch.bfloat16).contiguous()
    D = torch.empty((M, N), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tt_selftest_tcgen05_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                      ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(D.cpu().numpy().astype(np.float64), a @ b.T)


def _small_sum():
    dims = [40, 50, 45, 60, 40, 55]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(110, j), dims, const_ranks(N, r)) for j, r in enumerate([6, 9, 4, 7])]
    return dims, N, Ys


@pytest.mark.parametrize("tol", [0.0, 1e-8])
def test_mixed_vs_fp64_path(tol):
    """Sum rank 26 > l = 20, so the result depends on the sketch, and the
    partial contractions of the mixed path (14-bit digits) perturb it: the two
    paths must agree in ranks and in rounding error (<= 1.1x), and the outputs
    differ only at the level of that perturbation."""
    dims, N, Ys = _small_sum()
    ell = const_ranks(N, 20)
    sk = synth.gaussian_tt(synth.rng_for(111), dims, ell)
    Yd, skd = [to_dev(Y) for Y in Ys], to_dev(sk)
    X64 = to_host(tt.tt_round_sum_rand(Yd, ell, sketch=skd, tol=tol, precision="fp64"))
    Xmx = to_host(tt.tt_round_sum_rand(Yd, ell, sketch=skd, tol=tol, precision="mixed"))
    assert O.ranks_of(Xmx) == O.ranks_of(X64)
    Ysum = O.block_sum(Ys)
    e64 = O.diff_norm(X64, Ysum) / O.norm(Ysum)
    emx = O.diff_norm(Xmx, Ysum) / O.norm(Ysum)
    assert emx <= 1.1 * e64, (emx, e64)
    assert O.diff_norm(Xmx, X64) <= 1e-2 * O.norm(X64)


@pytest.mark.parametrize("tol,bound", [(0.0, 1e-8), (1e-12, 1e-11)])
def test_mixed_exact_recovery_when_sketch_covers_rank(tol, bound):
    """l = 30 >= sum rank 26: whatever the rounding of the sketch contractions,
    the sketched cores keep the whole range, so the mixed path reproduces the
    sum to the accuracy of its core updates: FP64 class in tolerance mode, the
    looser FP32-class target of the fixed-rank mode otherwise."""
    dims, N, Ys = _small_sum()
    ell = const_ranks(N, 30)
    Xmx = to_host(tt.tt_round_sum_rand([to_dev(Y) for Y in Ys], ell, seed=3, tol=tol, precision="mixed"))
    Ysum = O.block_sum(Ys)
    assert O.diff_norm(Xmx, Ysum) <= bound * O.norm(Ysum)


def _gate(Ys, ell, tol, seed=5):
    dims = [c.shape[1] for c in Ys[0]]
    sk = O.gaussian_sketch_philox(seed, dims, ell)
    Yd = [to_dev(Y) for Y in Ys]
    Xmx = to_host(tt.tt_round_sum_rand(Yd, ell, seed=seed, tol=tol, precision="mixed"))
    Xo = O.truncate_left_orthogonal(O.round_sum_randorth(Ys, sk), tol)
    Ysum = O.block_sum(Ys)
    e_or = O.diff_norm(Xo, Ysum) / O.norm(Ysum)
    e_mx = O.diff_norm(Xmx, Ysum) / O.norm(Ysum)
    return e_mx, e_or, Xmx, Xo


def test_mixed_accuracy_gate_structured_small():
    Ys = synth.workload_sum_structured(6, K=8, N=10, I=30, R=5, m=2, p=2, delta=1e-10)
    e_mx, e_or, Xmx, Xo = _gate(Ys, const_ranks(10, 14), 1e-8)
    assert O.ranks_of(Xmx) == O.ranks_of(Xo)
    assert e_mx <= 1.1 * e_or, (e_mx, e_or)


@pytest.mark.parametrize("form", ["structured", "literal"])
def test_mixed_accuracy_gate_full_size(form):
    """The benchmark workload (20 summands, N = 50, I = 100, rank 10, l = 30,
    tol 1e-8): mixed rounding error within 1.1x of the oracle's."""
    Ys = synth.workload_sum_structured(1, delta=1e-10) if form == "structured" else synth.workload_sum_literal(1)
    e_mx, e_or, Xmx, Xo = _gate(Ys, const_ranks(50, 30), 1e-8, seed=7)
    assert O.ranks_of(Xmx) == O.ranks_of(Xo)
    assert e_mx <= 1.1 * e_or, (e_mx, e_or)

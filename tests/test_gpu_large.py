"""Large sums: K = 30 summands, N = 30, I = 256, rank 20 (formal rank 600).
The structured redundant sum of Section 4.2's kind (three base TTs copied with
scrambled gauges and random coefficients, plus two summands of relative size
1e-8) is rounded at tolerance 1e-6 by Randomize-then-Orthogonalize (Algorithm
7 with the Section 3.2 truncation, sketch rank 70) in both precisions, and by
Two-Sided randomization (Algorithm 6, ranks 70 / 105) in both precisions. The oracle is far too
slow at this size, so the checks are properties that hold at any size, taken
on the GPU with blockwise TT inner products: the rounding error
||X - Y|| / ||Y|| stays within the tolerance, both precisions find the same
ranks, and the mixed path's error matches the FP64 one up to the resolution
of the inner-product formula (~1e-7 relative)."""
import numpy as np
import pytest
import torch

import synth
from tests._gpu import to_dev

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu

K, N, I, R, ELL, RHO, TOL = 30, 30, 256, 20, 70, 105, 1e-6


def _stack(Ys, n):
    return torch.stack([Y[n] for Y in Ys])            # (K, r0, I, r1): every summand has the same ranks


def _norm2_sum(Ys):
    W = torch.ones((len(Ys), len(Ys), 1, 1), dtype=torch.float64, device=Ys[0][0].device)
    for n in range(len(Ys[0])):
        A = _stack(Ys, n)
        W = torch.einsum("abij,aikr,bjks->abrs", W, A, A)
    return float(W.sum())


def _cross(X, Ys):
    W = torch.ones((len(Ys), 1, 1), dtype=torch.float64, device=X[0].device)
    for n in range(len(X)):
        W = torch.einsum("aij,ikr,ajks->ars", W, X[n], _stack(Ys, n))
    return float(W.sum())


def _norm2(X):
    W = torch.ones((1, 1), dtype=torch.float64, device=X[0].device)
    for c in X:
        W = torch.einsum("ij,ikr,jks->rs", W, c, c)
    return float(W.sum())


def _rel_err(X, Ys, y2):
    e2 = _norm2(X) - 2.0 * _cross(X, Ys) + y2
    return float(np.sqrt(max(e2, 0.0) / y2))


@pytest.fixture(scope="module")
def large_sum():
    Ys = synth.workload_sum_structured(5, K=K, N=N, I=I, R=R, m=3, p=2, delta=1e-8)
    Yd = [to_dev(Y) for Y in Ys]
    return Yd, _norm2_sum(Yd)


def test_large_sum_randorth_both_precisions(large_sum):
    Yd, y2 = large_sum
    ell = [1] + [ELL] * (N - 1) + [1]
    X64 = tt.tt_round_sum_rand(Yd, ell, seed=3, tol=TOL, precision="fp64")
    Xmx = tt.tt_round_sum_rand(Yd, ell, seed=3, tol=TOL, precision="mixed")
    r64 = [int(c.shape[0]) for c in X64] + [1]
    rmx = [int(c.shape[0]) for c in Xmx] + [1]
    assert r64 == rmx
    assert max(r64) <= ELL and max(r64) >= 3 * R      # the three bases span rank 60 at every inner bond
    e64, emx = _rel_err(X64, Yd, y2), _rel_err(Xmx, Yd, y2)
    assert e64 <= TOL and emx <= TOL, (e64, emx)
    assert emx <= 1.1 * e64 + 1e-7, (e64, emx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_sum_twosided(large_sum, precision):
    Yd, y2 = large_sum
    ell = [1] + [ELL] * (N - 1) + [1]
    rho = [1] + [RHO] * (N - 1) + [1]
    X = tt.tt_round_twosided(Yd, ell, rhos=rho, seed=4, precision=precision)
    assert [int(c.shape[0]) for c in X] == ell[:-1]
    e = _rel_err(X, Yd, y2)
    assert e <= TOL, e

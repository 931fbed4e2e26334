"""GPU parity of the TT arithmetic around the rounding (Section 2.3 inner
products and norms, the Section 4.2 operator's mode products and Gram-Schmidt
step) and of the synthetic TT-GMRES driver with the oracle's TT-GMRES on the
same seeds."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt
from paper_2110_04393_gb300 import gmres as G

pytestmark = pytest.mark.gpu


def test_inner_and_norm_match_oracle():
    dims = [7, 9, 8, 6, 7]
    X = synth.gaussian_tt(synth.rng_for(400), dims, [1, 3, 4, 5, 2, 1])
    Ys = [synth.gaussian_tt(synth.rng_for(401, j), dims, const_ranks(5, r)) for j, r in enumerate([2, 6, 3])]
    got = tt.tt_inner(to_dev(X), [to_dev(Y) for Y in Ys]).cpu().numpy()
    ref = np.array([O.inner(X, Y) for Y in Ys])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * O.norm(X) * max(O.norm(Y) for Y in Ys))
    assert abs(float(tt.tt_norm(to_dev(X))) - O.norm(X)) <= 1e-13 * O.norm(X)


def test_mode_products_match_oracle():
    dims = [6, 5, 7]
    Y = synth.gaussian_tt(synth.rng_for(402), dims, [1, 3, 4, 1])
    rng = synth.rng_for(403)
    mats = [rng.standard_normal((9, 6)), None, rng.standard_normal((7, 7))]
    ref = O.apply_term(Y, mats)
    Yd = to_dev(Y)
    out = tt.tt_mode_products([torch.from_numpy(mats[0]).cuda(), torch.from_numpy(mats[2]).cuda()], [Yd[0], Yd[2]])
    np.testing.assert_allclose(out[0].cpu().numpy(), ref[0], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out[1].cpu().numpy(), ref[2], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("k", [0, 1, 4])
def test_gram_schmidt_step_matches_oracle(k):
    dims = [8, 6, 7, 6, 8]
    N = len(dims)
    basis = []
    for j in range(k):
        V = synth.gaussian_tt(synth.rng_for(410, j), dims, const_ranks(N, 3))
        basis.append(synth.scale_tt(V, 1.0 / O.norm(V)))
    W = synth.gaussian_tt(synth.rng_for(411), dims, const_ranks(N, 4))
    ell = O.sum_sketch_ranks([W] + basis, 40)
    Vo, ho = O.gram_schmidt_round(W, basis, 40, 1e-10, 21)
    Vg, hg = tt.tt_round_gram_schmidt(to_dev(W), [to_dev(V) for V in basis], ell, tol=1e-10, seed=21)
    np.testing.assert_allclose(hg, ho, rtol=1e-11, atol=1e-13)
    Vg = to_host(Vg)
    assert O.ranks_of(Vg) == O.ranks_of(Vo)
    assert O.diff_norm(Vg, Vo) <= 1e-10
    assert abs(O.norm(Vg) - 1.0) <= 1e-12


def _terms_dev(op):
    return [[None if m is None else torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in t] for t in op["terms"]]


def test_tt_gmres_matches_oracle_gmres():
    op = synth.cookie_operator(N=4, I1=24, I=6)
    Minv = np.linalg.inv(sum(t[0] for t in op["terms"]))
    xo, ro, _ = O.tt_gmres(op["terms"], Minv, op["f"], tol=1e-8, maxit=30, ell_cap=40, seed0=500)
    xg, rg, ranks = G.tt_gmres(_terms_dev(op), torch.from_numpy(Minv).cuda(), to_dev(op["f"]), tol=1e-8, maxit=30,
                               ell_cap=40, seed0=500)
    assert len(rg) == len(ro) and rg[-1] <= 1e-8
    np.testing.assert_allclose(rg, ro, rtol=1e-5)
    xg = to_host(xg)
    assert O.ranks_of(xg) == O.ranks_of(xo)
    assert O.diff_norm(xg, xo) <= 1e-9 * O.norm(xo)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tt_gmres_paper_order_true_residual(precision):
    """N = 5 as in Section 4.2: the GPU solution's true residual
    ||f - A x|| / ||f|| (full tensors on the host) is that of the oracle's
    TT-GMRES on the same seeds (inexact Krylov: the roundings at 1e-9 leave a
    true residual above the 1e-8 estimate; both must agree)."""
    op = synth.cookie_operator(N=5, I1=40, I=8)
    Minv = np.linalg.inv(sum(t[0] for t in op["terms"]))
    f = O.full(op["f"])

    def true_res(x):
        Ax = sum(O.full(O.apply_term(x, t)) for t in op["terms"])
        return np.linalg.norm(f - Ax) / np.linalg.norm(f)

    xo, ro, _ = O.tt_gmres(op["terms"], Minv, op["f"], tol=1e-8, maxit=40, ell_cap=40, seed0=700)
    xg, rg, ranks = G.tt_gmres(_terms_dev(op), torch.from_numpy(Minv).cuda(), to_dev(op["f"]), tol=1e-8, maxit=40,
                               ell_cap=40, seed0=700, precision=precision)
    assert rg[-1] <= 1e-8
    eo, eg = true_res(xo), true_res(to_host(xg))
    assert eo < 1e-6
    assert eg <= (1.1 if precision == "fp64" else 2.0) * eo + 1e-9, (eg, eo)

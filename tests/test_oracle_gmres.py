"""Pins of the oracle's Section 4.2 pieces (TT-GMRES and its Gram-Schmidt
step) against dense linear algebra on full tensors."""
import numpy as np

import oracle as O
import synth


def _dense_operator(terms, dims):
    A = np.zeros((int(np.prod(dims)),) * 2)
    for t in terms:
        M = np.ones((1, 1))
        for n, m in enumerate(t):
            M = np.kron(M, m if m is not None else np.eye(dims[n]))
        A += M
    return A


def test_apply_term_is_the_kronecker_product():
    dims = [4, 3, 5]
    Y = synth.gaussian_tt(synth.rng_for(300), dims, [1, 2, 3, 1])
    rng = synth.rng_for(301)
    mats = [rng.standard_normal((4, 4)), None, rng.standard_normal((5, 5))]
    got = O.full(O.apply_term(Y, mats)).reshape(-1)
    K = np.kron(np.kron(mats[0], np.eye(3)), mats[2])
    np.testing.assert_allclose(got, K @ O.full(Y).reshape(-1), rtol=1e-12, atol=1e-12)


def test_gram_schmidt_step_orthonormalizes_and_reconstructs():
    """Exact case (sketch ranks above the true ranks, tiny tolerance): the new
    vector is orthonormal to the basis, the h are the dense inner products, and
    W = sum_j h_j V_j + h_{k+1} V_{k+1} on full tensors."""
    dims = [5, 4, 5, 4]
    N = len(dims)
    basis = []
    for j in range(3):
        V = synth.gaussian_tt(synth.rng_for(310, j), dims, [1, 2, 3, 2, 1])
        basis.append(synth.scale_tt(V, 1.0 / O.norm(V)))
    W = synth.gaussian_tt(synth.rng_for(311), dims, [1, 3, 2, 3, 1])
    Vn, h = O.gram_schmidt_round(W, basis, ell_cap=40, tol=1e-13, seed=5)
    Wf = O.full(W).reshape(-1)
    for j, V in enumerate(basis):
        assert abs(h[j] - float(O.full(V).reshape(-1) @ Wf)) <= 1e-12 * np.linalg.norm(Wf)
    assert abs(O.norm(Vn) - 1.0) <= 1e-12
    rec = sum(h[j] * O.full(V).reshape(-1) for j, V in enumerate(basis)) + h[-1] * O.full(Vn).reshape(-1)
    assert np.linalg.norm(rec - Wf) <= 1e-11 * np.linalg.norm(Wf)


def test_gram_schmidt_step_against_an_orthonormal_basis():
    """With an orthonormal basis (built by the step itself) the new vector is
    orthogonal to every basis vector: classical Gram-Schmidt in exact arithmetic."""
    dims = [5, 4, 5, 4]
    W0 = synth.gaussian_tt(synth.rng_for(312), dims, [1, 2, 2, 2, 1])
    basis = [synth.scale_tt(W0, 1.0 / O.norm(W0))]
    for j in range(3):
        W = synth.gaussian_tt(synth.rng_for(313, j), dims, [1, 2, 3, 2, 1])
        Vn, h = O.gram_schmidt_round(W, basis, ell_cap=60, tol=1e-14, seed=6 + j)
        basis.append(Vn)
    G = np.array([[O.inner(a, b) for b in basis] for a in basis])
    assert np.abs(G - np.eye(len(basis))).max() <= 1e-10


def test_tt_gmres_solves_the_synthetic_cookie_system():
    op = synth.cookie_operator(N=3, I1=12, I=5)
    dims, terms, f = op["dims"], op["terms"], op["f"]
    Minv = np.linalg.inv(sum(t[0] for t in terms))
    x, res, R = O.tt_gmres(terms, Minv, f, tol=1e-9, maxit=40, ell_cap=60)
    A = _dense_operator(terms, dims)
    xd = np.linalg.solve(A, O.full(f).reshape(-1))
    xt = O.full(x).reshape(-1)
    assert res[-1] <= 1e-9
    assert all(b <= a * (1 + 1e-6) for a, b in zip(res, res[1:]))
    assert np.linalg.norm(xt - xd) <= 1e-7 * np.linalg.norm(xd)
    r = O.full(f).reshape(-1) - A @ xt
    assert np.linalg.norm(r) <= 1e-7 * np.linalg.norm(O.full(f).reshape(-1))

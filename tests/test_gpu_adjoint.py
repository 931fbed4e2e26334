"""Hand-written adjoint of fixed-sketch RandOrth (tt_round_rand_backward and the
autograd Function) against the oracle's FP64 adjoint and against central
finite differences (h = 1e-6, FP64) of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle.adjoint import randorth_adjoint, randorth_fixed_sketch_loss, _environments
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu


def _case(N, I, R, ell, rT, seed):
    dims = [I] * N
    Y = synth.gaussian_tt(synth.rng_for(seed, 0), dims, const_ranks(N, R))
    el = tt.clamp_ranks(dims, const_ranks(N, ell))
    Om = synth.gaussian_tt(synth.rng_for(seed, 1), dims, el)
    T = synth.gaussian_tt(synth.rng_for(seed, 2), dims, const_ranks(N, rT))
    return dims, Y, el, Om, T


def _rel(a, b):
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return (num / den) ** 0.5


def _inner_torch(X, T):
    E = torch.ones((1, 1), dtype=torch.float64, device=X[0].device)
    for x, t in zip(X, T):
        E = torch.einsum("ab,aic,bid->cd", E, x, t)
    return E[0, 0]


@pytest.mark.parametrize("N,I,R,ell,rT", [(16, 32, 64, 16, 8), (5, 6, 4, 3, 2), (2, 7, 3, 2, 2)])
def test_backward_matches_oracle_adjoint(N, I, R, ell, rT):
    dims, Y, el, Om, T = _case(N, I, R, ell, rT, 40 + N)
    Yd, Omd = to_dev(Y), to_dev(Om)
    Xh = to_host(tt.tt_round_rand(Yd, el, sketch=Omd, tol=0.0))
    EL, ER = _environments(Xh, T)
    Xbar = [np.einsum("ac,cid,bd->aib", EL[n], T[n], ER[n + 1]) for n in range(N)]
    Yb = to_host(tt.tt_round_rand_backward(Yd, el, Omd, to_dev(Xbar)))
    Yo = randorth_adjoint(Y, Om, T)
    assert [y.shape for y in Yb] == [y.shape for y in Y]
    assert _rel(Yb, Yo) <= 1e-10


def test_autograd_function_matches_oracle():
    N, I, R, ell, rT = 6, 8, 5, 3, 2
    dims, Y, el, Om, T = _case(N, I, R, ell, rT, 77)
    cores = [torch.from_numpy(c).cuda().requires_grad_(True) for c in Y]
    Td = to_dev(T)
    X = tt.round_rand_fixed_sketch(cores, el, to_dev(Om))
    L = _inner_torch(X, Td)
    L.backward()
    Lv = float(L.detach())
    assert abs(Lv - randorth_fixed_sketch_loss(Y, Om, T)) <= 1e-12 * max(1.0, abs(Lv))
    g = [c.grad.cpu().numpy() for c in cores]
    assert _rel(g, randorth_adjoint(Y, Om, T)) <= 1e-10


def test_directional_central_difference():
    N, I, R, ell, rT = 6, 8, 5, 3, 2
    dims, Y, el, Om, T = _case(N, I, R, ell, rT, 91)
    Omd, Td = to_dev(Om), to_dev(T)
    rng = np.random.default_rng(5)
    for trial in range(3):
        Vd = [rng.standard_normal(c.shape) for c in Y]
        h = 1e-6

        def L(sign):
            Yp = [torch.from_numpy(c + sign * h * v).cuda() for c, v in zip(Y, Vd)]
            return float(_inner_torch(tt.tt_round_rand(Yp, el, sketch=Omd, tol=0.0), Td))

        fd = (L(1.0) - L(-1.0)) / (2 * h)
        cores = [torch.from_numpy(c).cuda() for c in Y]
        Xh = to_host(tt.tt_round_rand(cores, el, sketch=Omd, tol=0.0))
        EL, ER = _environments(Xh, T)
        Xbar = [np.einsum("ac,cid,bd->aib", EL[n], T[n], ER[n + 1]) for n in range(N)]
        g = to_host(tt.tt_round_rand_backward(cores, el, Omd, to_dev(Xbar)))
        an = sum(float(np.sum(a * v)) for a, v in zip(g, Vd))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (trial, fd, an)

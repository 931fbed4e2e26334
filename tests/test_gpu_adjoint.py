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


# ------------------------------------------------------------- float32 (cfg 4)

def _f32(cores):
    return [torch.from_numpy(np.ascontiguousarray(c, dtype=np.float32)).cuda() for c in cores]


def _as64(cores):
    return [np.asarray(c, dtype=np.float32).astype(np.float64) for c in cores]


def test_f32_forward_and_adjoint_at_cfg4_size():
    """N = 16, I = 32, R = 64 rounded to l = 16 with float32 storage: the
    forward and the adjoint within 1e-4 of the oracle's FP64 results on the
    same (float32-rounded) inputs and sketch."""
    N, I, R, ell, rT = 16, 32, 64, 16, 8
    dims, Y, el, Om, T = _case(N, I, R, ell, rT, 140)
    Y32, Om32 = _as64(Y), _as64(Om)
    Xg = tt.tt_round_rand(_f32(Y), el, sketch=_f32(Om), tol=0.0)
    assert all(c.dtype == torch.float32 for c in Xg)
    Xg64 = [c.double().cpu().numpy() for c in Xg]
    Xo = O.round_randorth(Y32, Om32)
    assert O.diff_norm(Xg64, Xo) <= 1e-4 * O.norm(Xo)
    # the cotangent of the GPU's own output cores (their QR gauge is the one the
    # backward recomputes; the gradient itself does not depend on the gauge)
    EL, ER = _environments(Xg64, T)
    Xbar = [np.einsum("ac,cid,bd->aib", EL[n], T[n], ER[n + 1]) for n in range(N)]
    Yb = tt.tt_round_rand_backward(_f32(Y), el, _f32(Om), _f32(Xbar))
    assert all(c.dtype == torch.float32 for c in Yb)
    Yo = randorth_adjoint(Y32, Om32, T)
    assert _rel([c.double().cpu().numpy() for c in Yb], Yo) <= 1e-4


def test_f32_autograd_and_directional_fd():
    N, I, R, ell, rT = 6, 8, 5, 3, 2
    dims, Y, el, Om, T = _case(N, I, R, ell, rT, 141)
    Y32, Om32 = _as64(Y), _as64(Om)
    cores = [c.requires_grad_(True) for c in _f32(Y)]
    X = tt.round_rand_fixed_sketch(cores, el, _f32(Om))
    Td = [c.float() for c in to_dev(T)]
    E = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    for x, t in zip(X, Td):
        E = torch.einsum("ab,aic,bid->cd", E, x, t)
    E[0, 0].backward()
    g = [c.grad.double().cpu().numpy() for c in cores]
    assert _rel(g, randorth_adjoint(Y32, Om32, T)) <= 1e-4
    # FP64 central differences (h = 1e-6) of the FP64 GPU forward on the rounded inputs
    Omd, Td64 = to_dev(Om32), to_dev(T)
    rng = np.random.default_rng(6)
    for trial in range(2):
        V = [rng.standard_normal(c.shape) for c in Y]
        h = 1e-6

        def L(sign):
            Yp = [torch.from_numpy(c + sign * h * v).cuda() for c, v in zip(Y32, V)]
            return float(_inner_torch(tt.tt_round_rand(Yp, el, sketch=Omd, tol=0.0), Td64))

        fd = (L(1.0) - L(-1.0)) / (2 * h)
        an = sum(float(np.sum(a * v)) for a, v in zip(g, V))
        assert abs(fd - an) <= 1e-4 * max(1.0, abs(fd)), (trial, fd, an)

"""GPU check of tt_round_sum_rand_noalloc, the entry point for callers that
cannot allocate device memory (it keeps its scratch in a fixed array inside the
library). Its result must match tt_round_sum_rand's on the same inputs and
precision (float64 and the mixed tensor-core path, whose emulated products use
extra regions of the array that must start at zero), on two calls in a row (the
second call reuses the array the first one left behind), without any device
allocation seen by the driver, and a problem too large for the array must be
refused with a clear message.

Runs last (file name) so that a failure here leaves every other test already
run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10   # the parity tolerance used by the other FP64 GPU tests


def _lib():
    from paper_2110_04393_gb300 import build, _native
    build.build()
    return _native.lib()


class _DeviceMemory:
    """Device-memory use seen by the CUDA driver: the free memory of the device
    (plain allocations) and the high-water mark of the device's default
    stream-ordered pool (cudaMallocAsync, which the workspace entry points use
    when given no workspace), reset on entry."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _pool_attr(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def snapshot(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return free.value, self._pool_attr(7)            # CU_MEMPOOL_ATTR_USED_MEM_CURRENT

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, 8, ctypes.byref(zero)) == 0   # USED_MEM_HIGH

    def high(self):
        return self._pool_attr(8)


def _call_noalloc(lib, Yd, ell, sk, coeffs, tol, precision, out):
    N, K = len(Yd[0]), len(Yd)
    dims = [int(c.shape[1]) for c in Yd[0]]
    ranks = [r for Y in Yd for r in ([int(Y[0].shape[0])] + [int(c.shape[2]) for c in Y])]
    i64 = lambda v: (ctypes.c_int64 * len(v))(*[int(x) for x in v])
    ptrs = lambda ts: (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    out_ranks = (ctypes.c_int64 * (N + 1))()
    co = (ctypes.c_double * K)(*coeffs)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tt_round_sum_rand_noalloc(N, K, i64(dims), i64(ranks), ptrs([c for Y in Yd for c in Y]), co, i64(ell),
                                       ptrs(sk), 0, float(tol), int(precision), ptrs(out), out_ranks, stream)
    assert rc == 0, lib.tt_last_error().decode()
    return list(out_ranks)


def _view(out, r, dims):
    return to_host([out[n].view(-1)[:r[n] * dims[n] * r[n + 1]].view(r[n], dims[n], r[n + 1])
                    for n in range(len(dims))])


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("tol", [0.0, 1e-6])
def test_noalloc_matches_workspace_entry_point_twice(tol, precision):
    import paper_2110_04393_gb300 as tt
    lib = _lib()
    dims = [24, 30, 28, 26, 24, 30, 22]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(70, j), dims, const_ranks(N, r)) for j, r in enumerate([5, 3, 6, 4])]
    ell = O.clamp_ranks(dims, const_ranks(N, 12))
    sk = synth.gaussian_tt(synth.rng_for(71), dims, ell)
    coeffs = [1.0, -0.75, 0.5, 2.0]
    Yd, skd = [to_dev(Y) for Y in Ys], to_dev(sk)
    ref = to_host(tt.tt_round_sum_rand(Yd, ell, sketch=skd, coeffs=coeffs, tol=tol,
                                       precision=["fp64", "mixed"][precision]))
    outs = [[torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device="cuda") for n in range(N)]
            for _ in range(2)]
    _call_noalloc(lib, Yd, ell, skd, coeffs, tol, precision, outs[0])    # first call: symbol look-up
    torch.cuda.synchronize()
    mem = _DeviceMemory()
    free0, used0 = mem.snapshot()
    mem.reset_high()
    torch_before = torch.cuda.memory_allocated()
    ranks = [_call_noalloc(lib, Yd, ell, skd, coeffs, tol, precision, outs[i]) for i in range(2)]
    torch.cuda.synchronize()
    free1, used1 = mem.snapshot()
    assert torch.cuda.memory_allocated() == torch_before
    assert used1 == used0 and mem.high() <= used0, "the call allocated from the stream-ordered pool"
    assert free1 == free0, "the call kept device memory"
    for i in range(2):
        got = _view(outs[i], ranks[i], dims)
        assert O.ranks_of(got) == O.ranks_of(ref)
        assert O.diff_norm(got, ref) <= FP64_TOL * O.norm(ref)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _lib()
    cap = lib.tt_noalloc_scratch_bytes()
    assert cap == 16 * 1024 * 1024
    N, K, I, R, l = 20, 12, 96, 16, 64
    dims = [I] * N
    Ys = [synth.gaussian_tt(synth.rng_for(72, j), dims, const_ranks(N, R)) for j in range(K)]
    ell = const_ranks(N, l)
    sk = synth.gaussian_tt(synth.rng_for(73), dims, ell)
    i64 = lambda v: (ctypes.c_int64 * len(v))(*v)
    ranks = [r for Y in Ys for r in const_ranks(N, R)]
    need = lib.tt_round_sum_rand_workspace(N, K, i64(dims), i64(ranks), i64(ell), 0.0, 0)
    assert need > cap
    Yd, skd = [to_dev(Y) for Y in Ys], to_dev(sk)
    out = [torch.empty((ell[n], dims[n], ell[n + 1]), dtype=torch.float64, device="cuda") for n in range(N)]
    with pytest.raises(AssertionError, match="above the fixed"):
        _call_noalloc(lib, Yd, ell, skd, [1.0] * K, 0.0, 0, out)

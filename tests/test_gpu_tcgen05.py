"""The tcgen05 tensor-core unit on its own: bf16 operands holding small
integers make every product and partial sum exact in fp32, so the GEMM must
reproduce the integer product bit for bit (this is also the exactness the
split FP64 GEMM relies on)."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 32, 128), (128, 48, 256), (257, 256, 64), (1000, 64, 192)])
def test_tcgen05_bf16_gemm_exact_on_integers(M, N, K):
    from paper_2110_04393_gb300 import _native
    lib = _native.lib()
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = rng.integers(-127, 128, size=(M, K)).astype(np.float64)
    b = rng.integers(-127, 128, size=(N, K)).astype(np.float64)
    A = torch.from_numpy(a).to("cuda", torch.bfloat16).contiguous()
    B = torch.from_numpy(b).to("cuda", torch.bfloat16).contiguous()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tt_selftest_tcgen05_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                      ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.tt_last_error().decode()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    np.testing.assert_array_equal(D.cpu().numpy().astype(np.float64), a @ b.T)

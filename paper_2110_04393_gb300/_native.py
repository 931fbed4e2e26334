"""Loader of the in-tree CUDA library (libttround.so). There is no CPU
fallback: importing a compute entry point without the library raises."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libttround.so")
_lib = None

c_i32, c_i64, c_u64, c_dbl, c_size, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                             ctypes.c_size_t, ctypes.c_void_p)
P_i64 = ctypes.POINTER(ctypes.c_int64)
P_dbl = ctypes.POINTER(ctypes.c_double)
P_vp = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes), mirroring include/ttround.h
SIGNATURES = {
    "tt_version": (ctypes.c_char_p, []),
    "tt_last_error": (ctypes.c_char_p, []),
    "tt_sketch_gaussian": (c_i32, [c_i32, P_i64, P_i64, c_u64, P_vp, c_vp]),
    "tt_round_sum_rand": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_vp, c_u64, c_dbl, c_i32,
                                  P_vp, P_i64, c_vp, c_size, c_vp]),
    "tt_round_sum_rand_workspace": (c_size, [c_i32, c_i32, P_i64, P_i64, P_i64, c_dbl, c_i32]),
    "tt_mixed_digits": (c_i32, [c_dbl, c_i32]),
    "tt_round_rand": (c_i32, [c_i32, P_i64, P_i64, P_vp, P_i64, P_vp, c_u64, c_dbl, c_i32, P_vp, P_i64, c_vp,
                              c_size, c_vp]),
    "tt_round_det": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, c_dbl, c_i64, P_vp, P_i64, c_vp, c_size,
                             c_vp]),
    "tt_round_det_workspace": (c_size, [c_i32, c_i32, P_i64, P_i64, c_dbl, c_i64]),
    "tt_round_det_out_capacity": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_i64]),
    "tt_round_orthrand": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_vp, c_u64, P_vp, P_i64, c_vp,
                                  c_size, c_vp]),
    "tt_round_orthrand_workspace": (c_size, [c_i32, c_i32, P_i64, P_i64, P_i64]),
    "tt_orthrand_omega_ranks": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_i64]),
    "tt_round_twosided": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_i64, P_vp, P_vp, c_u64, c_i32,
                                  P_vp, P_i64, c_vp, c_size, c_vp]),
    "tt_round_twosided_workspace": (c_size, [c_i32, c_i32, P_i64, P_i64, P_i64, P_i64, c_i32]),
    "tt_round_twosided_orth": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_i64, P_vp, P_vp, c_u64,
                                       c_dbl, c_i32, P_vp, P_i64, c_vp, c_size, c_vp]),
    "tt_round_twosided_orth_workspace": (c_size, [c_i32, c_i32, P_i64, P_i64, P_i64, P_i64, c_dbl, c_i32]),
    "tt_truncate_lorth": (c_i32, [c_i32, P_i64, P_i64, P_vp, c_dbl, c_i64, P_i64, c_vp, c_size, c_vp]),
    "tt_truncate_lorth_workspace": (c_size, [c_i32, P_i64, P_i64, c_dbl, c_i64]),
    "tt_inner": (c_i32, [c_i32, P_i64, P_i64, P_vp, c_i32, P_i64, P_vp, c_vp, c_vp, c_size, c_vp]),
    "tt_inner_workspace": (c_size, [c_i32, P_i64, P_i64, c_i32, P_i64]),
    "tt_norm": (c_i32, [c_i32, P_i64, P_i64, P_vp, c_vp, c_vp, c_size, c_vp]),
    "tt_norm_workspace": (c_size, [c_i32, P_i64, P_i64]),
    "tt_round_gram_schmidt": (c_i32, [c_i32, P_i64, P_i64, P_vp, c_i32, P_i64, P_vp, P_i64, P_vp, c_u64, c_dbl,
                                      c_i32, P_vp, P_i64, P_dbl, c_vp, c_size, c_vp]),
    "tt_round_gram_schmidt_workspace": (c_size, [c_i32, P_i64, P_i64, c_i32, P_i64, P_i64, c_dbl, c_i32]),
    "tt_mode_products": (c_i32, [c_i32, P_i64, P_vp, P_vp, P_vp, c_vp, c_size, c_vp]),
    "tt_mode_products_workspace": (c_size, [c_i32, P_i64]),
    "tt_round_sum_rand_sharded": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_vp, c_u64, c_dbl,
                                          c_i32, P_vp, P_i64, c_vp, c_size, c_vp, c_vp, c_vp]),
    "tt_noalloc_scratch_bytes": (c_size, []),
    "tt_round_sum_rand_noalloc": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_vp, P_dbl, P_i64, P_vp, c_u64, c_dbl,
                                          c_i32, P_vp, P_i64, c_vp]),
    "tt_round_rand_backward": (c_i32, [c_i32, P_i64, P_i64, P_vp, P_i64, P_vp, P_vp, P_vp, c_vp, c_size, c_vp]),
    "tt_round_rand_backward_workspace": (c_size, [c_i32, P_i64, P_i64, P_i64]),
    "tt_round_rand_f32": (c_i32, [c_i32, P_i64, P_i64, P_vp, P_i64, P_vp, c_u64, c_dbl, c_i32, P_vp, P_i64, c_vp,
                                  c_size, c_vp]),
    "tt_round_rand_f32_workspace": (c_size, [c_i32, P_i64, P_i64, P_i64, c_dbl, c_i32]),
    "tt_round_rand_backward_f32": (c_i32, [c_i32, P_i64, P_i64, P_vp, P_i64, P_vp, P_vp, P_vp, c_vp, c_size, c_vp]),
    "tt_round_rand_backward_f32_workspace": (c_size, [c_i32, P_i64, P_i64, P_i64]),
    "tt_sum_plan_create": (c_i32, [c_i32, c_i32, P_i64, P_i64, P_i64, c_dbl, c_i32, P_vp, c_vp]),
    "tt_sum_plan_run": (c_i32, [c_vp, P_vp, P_dbl, c_u64, P_vp, P_i64, c_vp]),
    "tt_sum_plan_destroy": (c_i32, [c_vp]),
    "tt_sum_plan_launches": (c_i64, [c_vp]),
    "tt_sum_plan_status": (c_i32, [c_vp, c_vp]),
    "tt_batch_plan_status": (c_i32, [c_vp, c_vp]),
    "tt_debug_inject_device_status": (None, [c_i32]),
    "tt_set_qr_mode": (c_i32, [c_i32]),
    "tt_set_gemm_mode": (c_i32, [c_i32]),
    "tt_tsqr_fallback_runs": (c_i32, [P_i64]),
    "tt_sum_plan_host_layout": (c_i32, [c_vp, P_i64, P_i64, P_i64, P_i64]),
    "tt_sum_plan_run_host": (c_i32, [c_vp, c_vp, P_dbl, c_u64, c_vp, P_i64, c_vp]),
    "tt_batch_plan_create": (c_i32, [c_i32, c_vp, c_i32, c_i32, P_vp, c_vp]),
    "tt_batch_plan_create_sched": (c_i32, [c_i32, c_vp, c_i32, c_vp, P_vp, c_vp]),
    "tt_batch_plan_is_fused": (c_i32, [c_vp]),
    "tt_batch_plan_run": (c_i32, [c_vp, P_vp, c_vp, P_vp, P_i64, c_vp]),
    "tt_batch_plan_destroy": (c_i32, [c_vp]),
    "tt_batch_plan_launches": (c_i64, [c_vp]),
    "tt_gemm_emulated_f64": (c_i32, [c_i64, c_i64, c_i64, c_dbl, c_vp, c_i64, c_i64, c_vp, c_i64, c_i64, c_dbl,
                                     c_vp, c_i64, c_i64, c_i32, c_vp, c_size, c_vp]),
    "tt_selftest_tcgen05_bf16": (c_i32, [c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tt_probe_fp64_rate": (c_i32, [c_i32, P_dbl, c_vp]),
    "tt_probe_pivot_rsqrt": (c_i32, [c_i64, P_i64, P_i64, c_vp]),
    "tt_prof_enable": (c_i32, [c_i32]),
    "tt_prof_reset": (c_i32, []),
    "tt_prof_read": (c_i32, [P_dbl, P_dbl, P_i64, P_i64]),
    "tt_prof_read_kind": (c_i32, [c_i32, P_dbl, P_dbl, P_i64]),
}


def lib():
    """The loaded library (raises RuntimeError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if hasattr(l, name):
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
        _lib = l
    return _lib


def last_error() -> str:
    return lib().tt_last_error().decode()

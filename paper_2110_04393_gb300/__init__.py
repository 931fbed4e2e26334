"""Randomized TT-rounding on GB300 (Al Daas et al., "Randomized algorithms for
rounding in the Tensor-Train format").

Python names mirror the C ABI of include/ttround.h. This layer only marshals
arguments: it checks and allocates torch CUDA tensors, passes raw device
pointers and the current CUDA stream, and reshapes the outputs. Every step of
the computation runs in the library's CUDA kernels; there is no fallback.

TT cores are torch.float64 CUDA tensors of shape (R_{n-1}, I_n, R_n),
C-contiguous.
"""
from __future__ import annotations

from .api import (tt_version, tt_sketch_gaussian, tt_round_sum_rand, tt_round_rand, TTError,
                  tt_round_det, tt_round_orthrand, tt_orthrand_omega_ranks, tt_round_twosided,
                  tt_round_twosided_orth, tt_truncate_lorth, tt_inner, tt_norm, tt_round_gram_schmidt,
                  tt_mode_products, tt_round_sum_rand_sharded,
                  tt_gemm_emulated_f64, SumRoundingPlan, BatchRoundingPlan, tune_batch_width, tune_batch_schedule, tt_round_rand_backward, clamp_ranks,
                  round_rand_fixed_sketch, debug_inject_device_status, set_qr_mode, tsqr_fallback_runs,
                  QR_AUTO, QR_CHAIN, QR_FORCE_FALLBACK, QR_COOP_THEN_FALLBACK, set_gemm_mode, GEMM_AUTO, GEMM_FUSED, GEMM_THREE_PASS, probe_fp64_rate, probe_pivot_rsqrt, prof_enable, prof_reset, prof_read, prof_read_kind,
                  PREC_FP64, PREC_MIXED)
from .costs import flops_sum_randorth, bytes_sum_randorth

__all__ = ["tt_version", "tt_sketch_gaussian", "tt_round_sum_rand", "tt_round_rand", "TTError",
           "tt_round_det", "tt_round_orthrand", "tt_orthrand_omega_ranks", "tt_round_twosided",
           "tt_round_twosided_orth", "tt_truncate_lorth", "tt_inner", "tt_norm", "tt_round_gram_schmidt",
           "tt_mode_products", "tt_round_sum_rand_sharded",
           "tt_gemm_emulated_f64", "SumRoundingPlan", "BatchRoundingPlan", "tune_batch_width", "tune_batch_schedule", "tt_round_rand_backward", "round_rand_fixed_sketch", "clamp_ranks",
           "PREC_FP64", "PREC_MIXED", "debug_inject_device_status", "set_qr_mode",
           "tsqr_fallback_runs", "QR_AUTO", "QR_CHAIN", "QR_FORCE_FALLBACK", "QR_COOP_THEN_FALLBACK", "set_gemm_mode",
           "GEMM_AUTO", "GEMM_FUSED", "GEMM_THREE_PASS", "probe_fp64_rate", "probe_pivot_rsqrt", "flops_sum_randorth", "bytes_sum_randorth"]

"""CPU FP64 oracle for randomized TT-rounding (Al Daas et al., "Randomized
algorithms for rounding in the Tensor-Train format").

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or calls
this package: only the tests, `__graft_entry__.smoke()` and the `cpu_baseline`
leg of `bench.py` (and its `--impl reference` arm) may use it. It shares no code
with the CUDA path; the two meet only in the seeded input generators of the
`synth` module.

Every function is a plain, slow NumPy restatement of the paper: the definitions
of Section 2 (unfoldings, TT sums, partial contractions) and the algorithms of
Sections 2.3 and 3 taken step by step in the paper's order and notation. A
library primitive (matmul, Householder QR, SVD) serves as one step; nothing is
blocked, fused or reordered beyond what the paper writes. Floating point is
float64 throughout.

Pins: tests/test_oracle_*.py check every function here against what the
mathematics fixes independently of this code (brute force on full tensors,
closed forms, invariants, exact recovery, textbook special cases).
Parity unpinned: none.
"""
from .tt import (H, V, from_H, from_V, full, full_bruteforce, inner, norm, diff_norm,
                 block_sum, merge_left, merge_right, ranks_of, dims_of)
from .rounding import (orthogonalize_rl, orthogonalize_lr, svd_truncated, tt_round_det,
                       partial_contractions_rl, partial_contractions_lr,
                       round_orthrand, round_randorth, round_twosided, round_sum_randorth, round_sum_randorth_sharded,
                       round_sum_twosided, round_sum_twosided_orth, truncate_left_orthogonal, clamp_ranks)
from .philox import philox4x32_10, gaussian_sketch_philox
from .adjoint import randorth_fixed_sketch_loss, randorth_adjoint
from .gmres import apply_term, gram_schmidt_round, tt_gmres, precondition, round_sum, sum_sketch_ranks

__all__ = [
    "H", "V", "from_H", "from_V", "full", "full_bruteforce", "inner", "norm", "diff_norm",
    "block_sum", "merge_left", "merge_right", "ranks_of", "dims_of",
    "orthogonalize_rl", "orthogonalize_lr", "svd_truncated", "tt_round_det",
    "partial_contractions_rl", "partial_contractions_lr",
    "round_orthrand", "round_randorth", "round_twosided", "round_sum_randorth", "round_sum_randorth_sharded",
    "round_sum_twosided", "round_sum_twosided_orth", "truncate_left_orthogonal", "clamp_ranks",
    "philox4x32_10", "gaussian_sketch_philox",
    "randorth_fixed_sketch_loss", "randorth_adjoint",
    "apply_term", "gram_schmidt_round", "tt_gmres", "precondition", "round_sum", "sum_sketch_ranks",
]

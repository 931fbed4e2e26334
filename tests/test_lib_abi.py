"""CPU checks of the C ABI: the library loads, exports every function that
include/ttround.h declares, rejects bad arguments before touching the GPU, and
the cost model reproduces the paper's flop table."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_04393_gb300 import build, _native
    build.build()
    return _native.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "ttround.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "tt_round_sum_rand" in names and "tt_round_rand" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ttround.h but not exported"


def test_python_signatures_cover_header(lib):
    from paper_2110_04393_gb300 import _native
    for n in _declared():
        assert n in _native.SIGNATURES, f"{n} has no ctypes signature"


def test_invalid_arguments_rejected_without_gpu(lib):
    i64 = lambda v: (ctypes.c_int64 * len(v))(*v)
    dims = i64([4, 4, 4])
    ells = i64([1, 2, 2, 1])
    bad_ranks = i64([2, 3, 3, 1])       # R_0 must be 1
    rc = lib.tt_round_sum_rand(3, 1, dims, bad_ranks, None, None, ells, None, 0, 0.0, 0, None, None, None, 0, None)
    assert rc == 1 and "ranks" in lib.tt_last_error().decode()
    rc = lib.tt_round_sum_rand(0, 1, dims, bad_ranks, None, None, ells, None, 0, 0.0, 0, None, None, None, 0, None)
    assert rc == 1
    big = i64([1, 2000, 2000, 1])
    ranks = i64([1, 3, 3, 1])
    sz = lib.tt_round_sum_rand_workspace(3, 1, i64([5000, 5000, 5000]), ranks, big, 0.0, 0)
    assert sz == 0 and "maximum" in lib.tt_last_error().decode()
    sz = lib.tt_round_sum_rand_workspace(3, 1, dims, ranks, ells, 0.0, 0)
    assert sz > 0


def test_cost_model_matches_paper_table():
    """Equal ranks: middle-core counts of the cost model equal the paper's
    Rand-then-Orth sum cost (Section 3.5.2) I (4 s R^2 l + 6 s R l^2 + 4 l^3)."""
    from paper_2110_04393_gb300.costs import flops_sum_randorth
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "cost_table.txt")):
        if line.strip() and not line.startswith("#"):
            name, *c = line.split()
            gold[name] = [float(x) for x in c]
    I, R, l, s = 37, 9, 5, 3
    N1, N2 = 10, 11
    dims1, dims2 = [I] * N1, [I] * N2
    Rs1 = [[1] + [R] * (N1 - 1) + [1]] * s
    Rs2 = [[1] + [R] * (N2 - 1) + [1]] * s
    e1 = [1] + [l] * (N1 - 1) + [1]
    e2 = [1] + [l] * (N2 - 1) + [1]
    per_core = flops_sum_randorth(dims2, Rs2, e2) - flops_sum_randorth(dims1, Rs1, e1)
    c = gold["Rand-then-Orth"]
    paper = I * (s * c[1] * R * R * l + s * c[2] * R * l * l + c[3] * l ** 3) - 4.0 * l ** 3 / 3
    assert abs(per_core - paper) <= 1e-9 * paper
    # with s = 1 it is the table's Rand-then-Orth row; Contr is its first part
    assert gold["Contr"] == [0, 2, 2, 0]


def test_mixed_digits_policy(lib):
    """Digits of the split tensor-core products: 2^(10 - 7 s) <= 1e-3 tol / N."""
    for tol in (1e-2, 1e-5, 1e-8, 1e-12):
        for N in (4, 50):
            s = lib.tt_mixed_digits(tol, N)
            target = 1e-3 * tol / N
            assert 1 <= s <= 8
            assert s == 8 or 2.0 ** (10 - 7 * s) <= target
            assert s == 1 or 2.0 ** (10 - 7 * (s - 1)) > target
    assert lib.tt_mixed_digits(1e-8, 50) == 8

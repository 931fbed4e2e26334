"""The algorithmic flop count behind every reported TFLOP/s, against Table 1's
per-core cost of Randomize-then-Orthogonalize for a sum (Section 3.5.2, reading
R11): each middle core costs I (4 s R^2 l + 6 s R l^2 + 4 l^3) for s summands of
rank R at sketch rank l, less the 4 l^3 / 3 that Householder's count subtracts.
The 20-TT benchmark sum (I = 100, R = 10, l = 30) gives 142.8 MFLOP per middle
core."""
import pytest

from paper_2110_04393_gb300.costs import flops_sum_randorth, bytes_sum_randorth


def _case(N, K=20, I=100, R=10, ell=30):
    dims = [I] * N
    ranks = [[1] + [R] * (N - 1) + [1] for _ in range(K)]
    ells = [1] + [ell] * (N - 1) + [1]
    return dims, ranks, ells


def test_middle_core_cost_is_table_1():
    # one more middle core (N -> N + 1) adds exactly one middle core's cost
    f50, f51 = flops_sum_randorth(*_case(50)), flops_sum_randorth(*_case(51))
    s, I, R, l = 20, 100, 10, 30
    table1 = I * (4 * s * R * R * l + 6 * s * R * l * l + 4 * l ** 3)
    assert table1 == 142.8e6
    assert f51 - f50 == pytest.approx(table1 - 4 * l ** 3 / 3, rel=1e-12)


def test_benchmark_totals():
    f = flops_sum_randorth(*_case(50))
    assert f == pytest.approx(6.858e9, rel=1e-3)            # 48 middle cores + 2 boundary cores
    b = bytes_sum_randorth(*_case(50))
    # inputs read twice, sketch and output once, float64
    dims, ranks, ells = _case(50)
    inp = sum(R[n] * dims[n] * R[n + 1] for R in ranks for n in range(50))
    assert inp * 8 == pytest.approx(77.12e6, rel=1e-6)       # the 77 MB of the benchmark's summands
    assert b == pytest.approx(223.4e6, rel=1e-3)

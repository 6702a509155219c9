"""bench.py's pure helpers on CPU: the roofline's algorithmic operation count,
the configuration object both arms print, and the FP64-rate fraction."""
import math

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402


@pytest.mark.parametrize("p", range(1, 9))
def test_algorithmic_count_is_the_dense_sum_factorised_form(p):
    # per direction a (p+1) x (p+1) matrix on each of the (p+1)^2 element lines
    # (p+1 outputs of p+1 multiply-adds, 2 flop each), plus 8 flop per node of
    # pointwise work
    n1 = p + 1
    lines, per_line = n1 * n1, 2 * n1 * n1
    assert bench.sem_flops_per_element(p) == 3 * lines * per_line + 8 * n1 ** 3


def test_headline_element_count():
    assert bench.sem_flops_per_element(7) == 28672


def test_both_arms_print_the_same_config():
    a = bench.bench_config()
    n = (7 * 16 + 1) ** 3
    assert a == bench.bench_config(n)
    assert a["nodes"] == 1442897 and a["elements"] == [16, 16, 16]
    assert a["p"] == 7 and a["s"] == 8 and a["tol"] == 1e-10
    assert a["workload"] == bench.workload_name()


def test_fp64_fraction_of_the_operation_rate():
    # as many node operations as the FP64 peak (2 per clock per SM) does in 1 ms
    ops_in_1ms = bench.FP64_PEAK_TFLOPS * 1e12 / 2 * 1e-3
    assert math.isclose(bench.fp64_frac(1, ops_in_1ms, 1.0), 1.0)
    assert math.isclose(bench.fp64_frac(2, ops_in_1ms, 4.0), 0.5)
    assert bench.fp64_frac(1, 10, 0) is None

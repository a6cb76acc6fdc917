"""The process-parallel evaluation of the oracle's sort-based forms
(oracle/parallel.py) against the serial forms it splits up, which the other
oracle pins tie to the paper: bit-exact on integers, within FP64 rounding on
floats (only the grouping of the sum over coordinates differs)."""
import numpy as np
import pytest

import oracle
from oracle import parallel
from paper_2210_15114_gb300 import inputs


@pytest.mark.parametrize("workers", [1, 3])
def test_l1_sort_parallel_equals_serial(workers):
    X = inputs.integer_points(5000, 7, 3, 0, 300)
    Z = inputs.integer_queries(5000, 4, 5)
    np.testing.assert_array_equal(parallel.l1_sort(X, Z, workers), oracle.l1_sort(X, Z))
    Xf = inputs.gaussian_mixture(5000, 7, 4, 2).astype(np.float32)
    Zf = inputs.gaussian_queries(5000, 4, 3)
    assert oracle.relative_error(parallel.l1_sort(Xf, Zf, workers), oracle.l1_sort(Xf, Zf)) <= 1e-14
    # one query column (1-D z) keeps its shape
    assert parallel.l1_sort(Xf, Zf[:, 0], workers).shape == (5000,)


def test_l1_grad_sort_parallel_equals_serial():
    X = inputs.integer_points(3000, 5, 4, 0, 50)         # many ties
    W = inputs.integer_queries(3000, 2, 6)
    Z = inputs.integer_queries(3000, 2, 7)
    np.testing.assert_array_equal(parallel.l1_grad_sort(X, W, Z, 3), oracle.l1_grad_sort(X, W, Z))


def test_lpp_odd_sort_parallel_equals_serial():
    X = inputs.integer_points(2000, 4, 8, -20, 20)
    Z = inputs.integer_queries(2000, 3, 9)
    np.testing.assert_array_equal(parallel.lpp_odd_sort(X, Z, 3, 2), oracle.lpp_odd_sort(X, Z, 3))
    with pytest.raises(ValueError):
        parallel.lpp_odd_sort(X, Z, 4)

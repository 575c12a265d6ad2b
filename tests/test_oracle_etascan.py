"""Pins of the oracle's reference-eta rule (Sec. 2): the largest eta of the converged range,
on hand-made metric sequences whose answer is fixed by the rule's definition."""
import numpy as np

from oracle import etascan


def _m(ft, it):
    m = np.zeros((len(ft), 5))
    m[:, 2] = ft
    m[:, 3] = it
    return m


def test_reference_is_the_end_of_the_converged_prefix():
    # F~(beta/2) within 1e-3 of the first value up to index 2; int F~ within 1e-3 everywhere
    m = _m([-1.0, -1.0005, -0.9991, -0.98, -1.0], [2.0, 2.001, 1.999, 2.0, 2.0])
    assert etascan.reference_eta(m, 1e-3) == 2
    # a later eta that returns inside the tolerance does not extend the range
    assert etascan.reference_eta(m, 3e-2) == 4
    assert etascan.reference_eta(m, 1e-4) == 0


def test_both_metrics_must_converge():
    m = _m([1.0, 1.0, 1.0, 1.0], [3.0, 3.0, 3.1, 3.0])
    assert etascan.reference_eta(m, 1e-3) == 1
    m = _m([1.0, 1.2, 1.0], [3.0, 3.0, 3.0])
    assert etascan.reference_eta(m, 1e-1) == 0


def test_single_eta():
    assert etascan.reference_eta(_m([0.5], [0.7]), 1e-6) == 0

"""Pins of the oracle's error metric and tolerances, the functions that decide
every parity verdict: ``rel_errors``, ``rel_errors_complex``,
``normwise_error`` and ``tolerance`` of the ``oracle`` package.

The metric is the componentwise one of the dot-product error bound,
e_ij = |c^_ij - c_ij| / (|A||B|)_ij, with exact equality required where the
normaliser is zero; the gates are 1e-6 sqrt(m) (FP32 accuracy), 1e-14 sqrt(m)
(FP64) and 2e-6 sqrt(m) (complex FP32).  Each ``pin_*`` takes a namespace that
holds the four functions (the oracle package itself, or a copy with one
planted mistake) and checks hand-worked values, so that a wrong constant, a
missing absolute value, sqrt(m) written as m, or a zero-normaliser branch
that forgives a difference fails at least one pin
(tests/test_oracle_metric.py plants those mistakes).
"""
from __future__ import annotations

import math

import numpy as np


def _eq(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (got.shape, want.shape)
    same = (got == want) | (np.isinf(got) & np.isinf(want) & (np.sign(got) == np.sign(want)))
    assert same.all(), (got.tolist(), want.tolist())


def pin_rel_errors_hand_worked(ns):
    """Hand-worked triples (c^, c, (|A||B|)) and their e."""
    c_hat = [1.0, 2.0, 3.0, -1.0, 0.0, -0.0, 1e-300, 5.0, 0.75]
    c_ref = [1.5, 2.0, 1.0, 1.0, 0.0, 0.0, 0.0, 5.0, 1.0]
    normr = [2.0, 4.0, 8.0, 4.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    want = [0.25,      # |1 - 1.5| / 2
            0.0,       # exact
            0.25,      # |3 - 1| / 8: the sign of the difference does not matter
            0.5,       # |-1 - 1| / 4
            0.0,       # zero normaliser, both zero
            0.0,       # zero normaliser, -0 == +0
            math.inf,  # zero normaliser, any difference at all
            0.0,       # zero normaliser, equal non-zero values
            0.5]       # |0.75 - 1| / 0.5
    _eq(ns.rel_errors(c_hat, c_ref, normr), want)
    # the normaliser divides: doubling it halves e
    _eq(ns.rel_errors([3.0], [1.0], [16.0]), [0.125])


def pin_rel_errors_nonfinite(ns):
    """A NaN or an infinity on either side is never within a tolerance."""
    c_hat = [math.nan, 1.0, math.inf, math.nan, math.inf]
    c_ref = [1.0, math.nan, 1.0, math.nan, math.inf]
    normr = [3.0, 3.0, 1.0, 1.0, 1.0]
    _eq(ns.rel_errors(c_hat, c_ref, normr), [math.inf] * 5)
    _eq(ns.rel_errors([math.nan], [0.0], [0.0]), [math.inf])


def pin_rel_errors_shapes(ns):
    """Elementwise over arrays, broadcasting nothing away."""
    c = np.arange(6.0).reshape(2, 3)
    e = ns.rel_errors(c + 0.5, c, np.full((2, 3), 2.0))
    _eq(e, np.full((2, 3), 0.25))
    assert ns.rel_errors(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3))).shape == (0, 3)


def pin_rel_errors_complex_hand_worked(ns):
    """Modulus of the complex difference over the modulus normaliser."""
    c_hat = [1 + 1j, 3 + 4j, 0j, 1j, 2 - 2j]
    c_ref = [1 + 0j, 0j, 0j, 0j, 2 - 2j]
    normr = [2.0, 10.0, 0.0, 0.0, 0.0]
    _eq(ns.rel_errors_complex(c_hat, c_ref, normr), [0.5, 0.5, 0.0, math.inf, 0.0])
    _eq(ns.rel_errors_complex([complex(math.nan, 0.0)], [1j], [1.0]), [math.inf])


def pin_normwise_hand_worked(ns):
    """max |c^ - c| / max |c|; the plain difference when c is all zero."""
    assert ns.normwise_error([1.0, 2.5], [1.0, 2.0]) == 0.25
    assert ns.normwise_error([1.0, -4.5], [1.0, -4.0]) == 0.125  # |c| of a negative entry
    assert ns.normwise_error([-3.0, 0.0], [1.0, 0.0]) == 4.0       # |c^ - c| of a sign flip
    assert ns.normwise_error([0.0, 0.5], [0.0, 0.0]) == 0.5
    assert ns.normwise_error(np.zeros((0, 4)), np.zeros((0, 4))) == 0.0


def pin_tolerance_literals(ns):
    """The stated gates as literal numbers."""
    close = lambda a, b: abs(a - b) <= 1e-12 * abs(b)
    assert close(ns.tolerance(256, "f32"), 1.6e-5)
    assert close(ns.tolerance(256, "split"), 1.6e-5)
    assert close(ns.tolerance(256, "simt"), 1.6e-5)
    assert close(ns.tolerance(4096, "f64"), 6.4e-13)
    assert close(ns.tolerance(4096, "dgemm"), 6.4e-13)
    assert close(ns.tolerance(100, "c32"), 2e-5)
    assert close(ns.tolerance(10000, "f32"), 1e-4)
    # m below 1 (m = 0 writes C = 0 exactly) is held to the m = 1 gate
    assert close(ns.tolerance(0, "f32"), 1e-6)
    assert close(ns.tolerance(1, "f64"), 1e-14)
    try:
        ns.tolerance(16, "fp8")
    except ValueError:
        pass
    else:
        raise AssertionError("FP8 has no gate: tolerance must refuse it")


ALL_METRIC_PINS = [pin_rel_errors_hand_worked, pin_rel_errors_nonfinite, pin_rel_errors_shapes,
                   pin_rel_errors_complex_hand_worked, pin_normwise_hand_worked,
                   pin_tolerance_literals]

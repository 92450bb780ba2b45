"""The oracle's error metric and tolerances against hand-worked values, and
planted mistakes in a copy of them that each pin must catch (runs without a
GPU).  The copy is made from the source text of ``oracle/__init__.py``'s
metric functions with one substitution each, so the pins are shown to catch
the mistakes a reader could plausibly make in those lines."""
import inspect
import types

import numpy as np
import pytest

import oracle
import metric_pins

FUNCS = ("rel_errors", "rel_errors_complex", "tolerance", "normwise_error")


def _namespace(replace=None):
    """A namespace holding the four metric functions, compiled from the
    oracle's own source with at most one (old, new) substitution."""
    src = "\n\n".join(inspect.getsource(getattr(oracle, f)) for f in FUNCS)
    if replace is not None:
        old, new = replace
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = {"np": np}
    exec(compile(src, "<metric>", "exec"), ns)
    return types.SimpleNamespace(**{f: ns[f] for f in FUNCS})


@pytest.mark.parametrize("pin", metric_pins.ALL_METRIC_PINS, ids=lambda f: f.__name__)
def test_metric_pin(pin):
    pin(oracle)


def test_copy_is_faithful():
    # the unmodified copy passes every pin, so a failure below is the mistake's
    for pin in metric_pins.ALL_METRIC_PINS:
        pin(_namespace())


MISTAKES = {
    "tolerance constant 1e-5": ("return 1e-6 * np.sqrt(m)", "return 1e-5 * np.sqrt(m)"),
    "tolerance m for sqrt(m)": ("return 1e-6 * np.sqrt(m)", "return 1e-6 * m"),
    "f64 constant 1e-13": ("return 1e-14 * np.sqrt(m)", "return 1e-13 * np.sqrt(m)"),
    "f64 m for sqrt(m)": ("return 1e-14 * np.sqrt(m)", "return 1e-14 * m"),
    "complex constant": ("return 2e-6 * np.sqrt(m)", "return 1e-6 * np.sqrt(m)"),
    "m not clamped": ("m = max(int(m), 1)", "m = int(m)"),
    "difference without abs": ("        diff = np.abs(c_hat - c_ref)\n",
                               "        diff = c_hat - c_ref\n"),
    "zero normaliser forgives": ("np.where(diff == 0, 0.0, np.inf))\n    return np.where(np.isnan(diff), np.inf, e)\n\n\ndef rel_errors_complex",
                                 "0.0)\n    return np.where(np.isnan(diff), np.inf, e)\n\n\ndef rel_errors_complex"),
    "NaN passes": ("    return np.where(np.isnan(diff), np.inf, e)\n\n\ndef rel_errors_complex",
                   "    return e\n\n\ndef rel_errors_complex"),
    "normaliser multiplies": ("        diff = np.abs(c_hat - c_ref)\n    with np.errstate(divide=\"ignore\", invalid=\"ignore\"):\n        e = np.where(abs_ref > 0, diff / np.where",
                              "        diff = np.abs(c_hat - c_ref)\n    with np.errstate(divide=\"ignore\", invalid=\"ignore\"):\n        e = np.where(abs_ref > 0, diff * np.where"),
    "complex without modulus": ("abs_ref = np.asarray(abs_ref, np.float64)\n    diff = np.abs(c_hat - c_ref)",
                                "abs_ref = np.asarray(abs_ref, np.float64)\n    diff = np.abs(np.real(c_hat - c_ref))"),
    "normwise without scaling": ("return d / mx if mx > 0 else d", "return d"),
    "normwise max without abs": ("mx = float(np.max(np.abs(c_ref)))", "mx = float(np.max(c_ref))"),
    "normwise diff without abs": ("d = float(np.max(np.abs(np.asarray(c_hat, np.float64) - c_ref)))",
                                  "d = float(np.max(np.asarray(c_hat, np.float64) - c_ref))"),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_is_caught(name):
    ns = _namespace(MISTAKES[name])
    failed = []
    for pin in metric_pins.ALL_METRIC_PINS:
        try:
            pin(ns)
        except (AssertionError, ValueError, TypeError):
            failed.append(pin.__name__)
    assert failed, "planted mistake %r passed every metric pin" % name

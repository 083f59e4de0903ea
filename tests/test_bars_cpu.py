"""The parity bars themselves: a check that the GPU tests' tolerance reading
(entry-wise relative with a 1e-3 floor for complex128, normwise for
complex64, variances relative to <H^2>) rejects what it should."""

import numpy as np
import pytest

import bars


def test_complex128_bar_is_relative_per_entry():
    want = np.array([1.0, 1e-2, -3e-3])
    # every entry off by 0.9 of its own bar passes
    got = want + 0.9 * 1e-10 * np.abs(want)
    assert bars.check(got, want, "c128", 1e-10, "e") == pytest.approx(0.9, rel=1e-3)
    # a small entry off by 2x its own relative bar fails, though the error is far
    # below the bar of the largest entry
    got = want.copy()
    got[1] += 2e-10 * 1e-2
    with pytest.raises(AssertionError, match="entry"):
        bars.check(got, want, "c128", 1e-10, "e")


def test_complex128_floor_is_a_thousandth_of_the_largest_entry():
    want = np.array([2.0, 0.0, 1e-9])
    got = want + np.array([0.0, 0.9e-10 * 2e-3, 0.9e-10 * 2e-3])  # below tol * 1e-3 * max
    assert bars.check(got, want, "c128", 1e-10, "e") < 1.0
    got[1] = 1.1e-10 * 2e-3
    with pytest.raises(AssertionError):
        bars.check(got, want, "c128", 1e-10, "e")


def test_double_float_is_held_to_the_complex128_bar():
    assert bars.TOL_E["c128df"] == bars.TOL_E["c128"] == 1e-10
    assert bars.TOL_J["c128df"] == bars.TOL_J["c128"] == 1e-9
    want = np.array([1.0, 1e-2])
    got = want + np.array([0.0, 2e-11])  # 2e-9 relative on the small entry
    with pytest.raises(AssertionError):
        bars.check_j(got, want, "c128df")


def test_complex64_bar_is_normwise():
    want = np.array([1.0, 1e-6, -0.5])
    got = want + np.array([0.0, 0.9e-4, 0.0])  # large relative error on a tiny entry: normwise passes
    assert bars.check_e(got, want, "c64") == pytest.approx(0.9, rel=1e-6)
    got[0] += 2e-4
    with pytest.raises(AssertionError):
        bars.check_e(got, want, "c64")


def test_variance_bar_scales_with_the_second_moment():
    var = np.array([1e-6])      # <H^2> - <H>^2, a small difference of large moments
    h2 = np.array([4.0])        # <H^2>
    got = var + 3e-10           # within 1e-10 * <H^2>, far outside 1e-10 * Var
    assert bars.check(got, var, "c128", 1e-10, "var", magnitude=h2) < 1.0
    with pytest.raises(AssertionError):
        bars.check(got, var, "c128", 1e-10, "var")


def test_shapes_must_match_and_empty_arrays_pass():
    with pytest.raises(AssertionError, match="shape"):
        bars.check(np.zeros(3), np.zeros(4), "c128", 1e-10, "e")
    assert bars.check(np.zeros(0), np.zeros(0), "c64", 1e-4, "e") == 0.0
    with pytest.raises(AssertionError):
        bars.check_state(np.array([1.0 + 2e-12j]), np.array([1.0 + 0j]), "c128")

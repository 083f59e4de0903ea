"""Parity bars of the CUDA path against the FP64 oracle.

The accuracy targets: complex128 results within 1e-10 relative on expectation
values and 1e-9 relative on gradients, complex64 results within 1e-4.  How the
bars are read (each reading follows from the arithmetic):

* complex128 (FP64 arithmetic, or double-float arithmetic with FP64
  reductions): entry by entry, relative to max(|x_i|, 1e-3 * max_j |x_j|).
  The floor keeps an entry that is zero or nearly so from demanding an
  error below the rounding of the array's large entries; above it every
  entry is held to the relative bar.
* complex64 (FP32 gate arithmetic, FP64 / compensated reductions): normwise,
  max_i |got_i - x_i| <= 1e-4 * max_j |x_j|.  FP32 rounding enters every
  amplitude at unit roundoff 6e-8 per gate, an absolute error in the scale of
  the whole array, not of each entry; a small entry carries the same
  absolute error as a large one.
* Variances Var = <H^2> - <H>^2 are formed as a difference, so their
  rounding error scales with <H^2>, not with Var: the bar is relative to
  <H^2> (entry by entry for complex128, normwise for complex64).
* Amplitudes: absolute, 1e-12 (complex128) and 1e-4 (complex64), the state
  having unit norm.
"""

from __future__ import annotations

import numpy as np

TOL_STATE = {"c128": 1e-12, "c64": 1e-4, "c128df": 1e-12}
TOL_E = {"c128": 1e-10, "c64": 1e-4, "c128df": 1e-10}
TOL_J = {"c128": 1e-9, "c64": 1e-4, "c128df": 1e-9}
FLOOR = 1e-3


def scale(want: np.ndarray, dtype: str) -> np.ndarray:
    """Per-entry magnitude the relative bar multiplies."""
    a = np.abs(np.asarray(want, dtype=np.float64))
    if a.size == 0:
        return a
    top = float(a.max())
    if dtype == "c64":
        return np.full_like(a, top)
    return np.maximum(a, FLOOR * top)


def check(got, want, dtype: str, tol: float, what: str, magnitude=None) -> float:
    """Assert the bar; return the largest error relative to it (<= 1 passes).

    ``magnitude``: the entries' own scale when it differs from |want| (the
    variance's <H^2>)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, f"{what}: shape {got.shape} != {want.shape}"
    if want.size == 0:
        return 0.0
    s = scale(want if magnitude is None else magnitude, dtype)
    err = np.abs(got - want)
    bar = tol * s
    ok = err <= bar
    if not np.all(ok):
        i = np.unravel_index(int(np.argmax(err - bar)), err.shape)
        raise AssertionError(f"{what} ({dtype}): entry {i} got {got[i]!r} want {want[i]!r} error {err[i]:.3e} "
                             f"> bar {bar[i]:.3e} ({int((~ok).sum())} of {ok.size} entries over)")
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bar > 0, err / np.where(bar > 0, bar, 1.0), 0.0)
    return float(r.max())


def check_e(got, want, dtype, what="expval"):
    return check(got, want, dtype, TOL_E[dtype], what)


def check_j(got, want, dtype, what="jacobian"):
    return check(got, want, dtype, TOL_J[dtype], what)


def check_state(got, want, dtype):
    err = float(np.abs(np.asarray(got).astype(np.complex128) - want).max()) if np.size(want) else 0.0
    assert err <= TOL_STATE[dtype], f"max amplitude error {err:.3e} > {TOL_STATE[dtype]:.0e} ({dtype})"
    return err


# measured errors of the parity checks, written out at the end of a session
# when SV_PARITY_REPORT names a file (tests/conftest.py)
RECORDS = []


def record(what: str, dtype: str, got, want, ratio: float) -> None:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    err = float(np.abs(got - want).max()) if want.size else 0.0
    RECORDS.append({"what": what, "dtype": dtype, "entries": int(want.size), "max_abs_error": err,
                    "max_abs_value": float(np.abs(want).max()) if want.size else 0.0,
                    "error_over_bar": ratio})

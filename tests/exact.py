"""Exact checks of |x - x'| <= e for the tests (rational arithmetic).

The bulk of the values is decided with float64 / longdouble arithmetic where
that is provably exact or far from the boundary; every value near the boundary
is re-decided with fractions.Fraction.
"""
from fractions import Fraction

import numpy as np


def exact_abs_diff_le(x, y, e):
    """Element-wise exact |x - y| <= e for finite float arrays x, y and scalar e.

    Returns a bool array.  Raises if any input is not finite.
    """
    x = np.asarray(x)
    y = np.asarray(y)
    assert x.shape == y.shape
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(y))
    xl = x.astype(np.longdouble)
    yl = y.astype(np.longdouble)
    d = np.abs(xl - yl)
    el = np.longdouble(e)
    # far from the boundary: decided (relative error of d is < 2^-60 at most
    # when the difference is not exact; 2^-40 leaves a wide margin)
    clear_yes = d < el * (1 - np.longdouble(2.0) ** -40)
    clear_no = d > el * (1 + np.longdouble(2.0) ** -40)
    out = clear_yes.copy()
    unsure = ~(clear_yes | clear_no)
    fe = Fraction(float(e))
    for i in np.flatnonzero(unsure.ravel()):
        a = Fraction(float(x.ravel()[i]))
        b = Fraction(float(y.ravel()[i]))
        out.ravel()[i] = abs(a - b) <= fe
    return out


def within_exact_scalar(a, b, e):
    return abs(Fraction(float(a)) - Fraction(float(b))) <= Fraction(float(e))

"""Oracle of Ng acceleration of the Lambda iteration (a fixed-point extrapolation; not in the
paper, which iterates plain Lambda, Sect. 2.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

From the last four iterates x0 (newest), x1, x2, x3 of a fixed-point iteration, with the
differences d0 = x0 - x1, d1 = x1 - x2, d2 = x2 - x3, choose a, b minimising the weighted norm of
d0 - a (d0 - d1) - b (d0 - d2) -- the next difference predicted by a recurrence of order two --
and take x = (1 - a - b) x0 + a x1 + b x2.  Weights 1/x0^2, so that every population counts by its
relative change.  If the iteration's error lies in a subspace on which the iteration matrix has at
most two eigenvalues, the predicted difference vanishes exactly and x is the fixed point.
"""
from __future__ import annotations

import numpy as np


def ng_coefficients(x0, x1, x2, x3, weights=None):
    """(a, b) of the second-order extrapolation."""
    x0, x1, x2, x3 = (np.asarray(v, float).ravel() for v in (x0, x1, x2, x3))
    w = 1.0 / x0 ** 2 if weights is None else np.asarray(weights, float).ravel()
    d0, d1, d2 = x0 - x1, x1 - x2, x2 - x3
    u, v = d0 - d1, d0 - d2
    A = np.array([[np.sum(w * u * u), np.sum(w * u * v)], [np.sum(w * u * v), np.sum(w * v * v)]])
    B = np.array([np.sum(w * d0 * u), np.sum(w * d0 * v)])
    return np.linalg.solve(A, B)


def ng_extrapolate(x0, x1, x2, x3, weights=None):
    a, b = ng_coefficients(x0, x1, x2, x3, weights)
    return (1.0 - a - b) * np.asarray(x0, float) + a * np.asarray(x1, float) + \
        b * np.asarray(x2, float)

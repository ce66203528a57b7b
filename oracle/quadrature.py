"""Quadrature rules of the oracle (test infrastructure).

Triangle rules are given in barycentric coordinates with weights summing to 1,
so that  int_tau f = |tau| * sum_k w_k f(x_k).

  * 6-point degree-4 rule (Dunavant 1985, two 3-point orbits) - the regular
    rule of the reference plan, matching the paper's "quadrature order 4"
    (Results, arginine benchmark) as read in the design notes.
  * 3-point degree-2 rule (points (1/6,1/6,2/3) and permutations) - the cheaper
    regular rule of a relaxed plan.
  * 1-point centroid rule (degree 1).

Gauss-Legendre nodes on [0,1] come from NumPy's ``leggauss`` (a library
routine), mapped affinely.
"""
import numpy as np

_A1, _W1 = 0.445948490915965, 0.223381589678011
_A2, _W2 = 0.091576213509771, 0.109951743655322


def _orbit3(a):
    b = 1.0 - 2.0 * a
    return [[b, a, a], [a, b, a], [a, a, b]]


def triangle_rule(q: int):
    """(barycentric points [q,3], weights [q]) of the q-point rule."""
    if q == 6:
        pts = np.array(_orbit3(_A1) + _orbit3(_A2), dtype=np.float64)
        w = np.array([_W1] * 3 + [_W2] * 3, dtype=np.float64)
    elif q == 3:
        pts = np.array(_orbit3(1.0 / 6.0), dtype=np.float64)
        w = np.full(3, 1.0 / 3.0)
    elif q == 1:
        pts = np.array([[1.0 / 3.0] * 3])
        w = np.ones(1)
    else:
        raise ValueError(f"no {q}-point triangle rule")
    return np.ascontiguousarray(pts), np.ascontiguousarray(w)


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return np.ascontiguousarray(0.5 * (x + 1.0)), np.ascontiguousarray(0.5 * w)

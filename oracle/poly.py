"""Minimal multivariate polynomials with float64 coefficients (oracle helper).

A polynomial in the variables C_0 .. C_{N-1} is a dict mapping an exponent
tuple of length N to its coefficient.  Only what the oracle needs to expand
the bulk flux potential of Sec. II into monomials is here: sums, products,
scaling, degree-wise homogenisation on the simplex sum_i C_i = 1, exact
division by one variable, and evaluation.
"""
from __future__ import annotations

import numpy as np


class Poly:
    __slots__ = ("n", "terms")

    def __init__(self, n, terms=None):
        self.n = n
        self.terms = dict(terms) if terms else {}

    @staticmethod
    def const(n, c):
        return Poly(n, {(0,) * n: float(c)}) if c != 0 else Poly(n)

    @staticmethod
    def var(n, i, c=1.0):
        e = [0] * n
        e[i] = 1
        return Poly(n, {tuple(e): float(c)})

    def copy(self):
        return Poly(self.n, self.terms)

    def __add__(self, other):
        if not isinstance(other, Poly):
            other = Poly.const(self.n, other)
        out = dict(self.terms)
        for e, c in other.terms.items():
            out[e] = out.get(e, 0.0) + c
        return Poly(self.n, out)

    __radd__ = __add__

    def __neg__(self):
        return Poly(self.n, {e: -c for e, c in self.terms.items()})

    def __sub__(self, other):
        if not isinstance(other, Poly):
            other = Poly.const(self.n, other)
        return self + (-other)

    def __rsub__(self, other):
        return (-self) + other

    def __mul__(self, other):
        if not isinstance(other, Poly):
            return Poly(self.n, {e: c * float(other) for e, c in self.terms.items()})
        out = {}
        for e1, c1 in self.terms.items():
            for e2, c2 in other.terms.items():
                e = tuple(a + b for a, b in zip(e1, e2))
                out[e] = out.get(e, 0.0) + c1 * c2
        return Poly(self.n, out)

    __rmul__ = __mul__

    def __pow__(self, k):
        out = Poly.const(self.n, 1.0)
        for _ in range(k):
            out = out * self
        return out

    def degree(self):
        return max((sum(e) for e in self.terms), default=0)

    def homogenise(self, degree):
        """Multiply each degree-d part by (sum_i C_i)^(degree - d).

        On the simplex sum_i C_i = 1 this leaves the polynomial's values
        unchanged and makes it homogeneous of the given degree.
        """
        s = Poly(self.n)
        for i in range(self.n):
            s = s + Poly.var(self.n, i)
        out = Poly(self.n)
        for e, c in self.terms.items():
            d = sum(e)
            if d > degree:
                raise ValueError("term of degree above the target")
            out = out + Poly(self.n, {e: c}) * (s ** (degree - d))
        return out

    def split_by_var(self, i):
        """(part divisible by C_i, divided by C_i;  part free of C_i)."""
        with_i, without_i = {}, {}
        for e, c in self.terms.items():
            if e[i] > 0:
                e2 = list(e)
                e2[i] -= 1
                with_i[tuple(e2)] = c
            else:
                without_i[e] = c
        return Poly(self.n, with_i), Poly(self.n, without_i)

    def max_abs_coeff(self):
        return max((abs(c) for c in self.terms.values()), default=0.0)

    def __call__(self, C):
        """Evaluate at C (shape (n, ...)); returns an array of shape C.shape[1:]."""
        C = np.asarray(C, dtype=np.float64)
        out = np.zeros(C.shape[1:])
        for e, c in self.terms.items():
            t = np.full(C.shape[1:], c)
            for i, k in enumerate(e):
                if k:
                    t = t * C[i] ** k
            out = out + t
        return out

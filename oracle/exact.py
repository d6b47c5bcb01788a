"""Eq. (1) in exact rational arithmetic -- TEST INFRASTRUCTURE ONLY.

For tiny inputs with rational entries this evaluates
b = (X^T M^{-1} X)^{-1} X^T M^{-1} y (Section 1, Eq. (1)) with Python fractions and
Gauss-Jordan elimination, so the result carries no rounding at all. It pins the
FP64 routes in ``oracle.gls`` (their difference must be a rounding error only).
Only ``tests/`` may import it.
"""
from __future__ import annotations

from fractions import Fraction


def _frac_matrix(A):
    return [[Fraction(v) for v in row] for row in A]


def inverse(A):
    """Exact inverse of a square rational matrix (list of lists) by Gauss-Jordan."""
    A = _frac_matrix(A)
    n = len(A)
    aug = [row + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next((r for r in range(col, n) if aug[r][col] != 0), None)
        if piv is None:
            raise ZeroDivisionError("singular matrix")
        aug[col], aug[piv] = aug[piv], aug[col]
        inv_p = 1 / aug[col][col]
        aug[col] = [v * inv_p for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * c for a, c in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


def matmul(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(len(B))) for j in range(len(B[0]))]
            for i in range(len(A))]


def transpose(A):
    return [list(r) for r in zip(*A)]


def gls_exact(M, X, y):
    """Exact (b, Wald) for one design matrix X (n x p) and one phenotype y (length n).

    Wald = b_p^2 / ((X^T M^{-1} X)^{-1})_pp, both returned as Fractions.
    """
    Mi = inverse(M)
    Xf = _frac_matrix(X)
    yf = [[Fraction(v)] for v in y]
    Xt = transpose(Xf)
    A = matmul(matmul(Xt, Mi), Xf)
    r = matmul(matmul(Xt, Mi), yf)
    Ai = inverse(A)
    b = [row[0] for row in matmul(Ai, r)]
    wald = b[-1] ** 2 / Ai[-1][-1]
    return b, wald

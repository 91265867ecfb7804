"""Oracle dense linear algebra (test infrastructure only).

* ``lu_factor`` / ``lu_solve``: unblocked Gaussian elimination with partial
  pivoting, one column at a time (the "standard LU factorization" §4.1 compares
  against).  Pivot = first row index maximising |Re| + |Im| (the LAPACK izamax
  convention; the paper does not fix a tie-break, so solutions, never pivots,
  are compared across implementations).
* ``schur_solve``: Theorem thm:LU and Corollary lem:for_ssm_RHS (§4.1):
      U33 = -M31 M13 - M32 M23,
      z3  = U33^{-1} (b3 - M31 b1 - M32 b2),
      x1  = b1 - M13 z3,  x2 = b2 - M23 z3,  x3 = z3.
  Matrix products use numpy's matmul (a library primitive).
* ``backward_error_*``: normwise backward error per right-hand side,
  eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), max over columns
  (the paper states no norm; this is the reading used for the 1e-9 target).
"""
from __future__ import annotations

import numpy as np


class SingularMatrix(Exception):
    def __init__(self, col: int):
        super().__init__(f"zero pivot in column {col}")
        self.col = col


def lu_factor_columns(A: np.ndarray):
    """The elimination of ``lu_factor`` one column at a time: a generator that yields the column
    index k after eliminating column k, and finally returns (LU, piv) (as StopIteration.value).
    The arithmetic is exactly lu_factor's; the generator form only lets a caller time or pause the
    factorisation between columns."""
    LU = np.array(A, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    piv = np.arange(n)
    for k in range(n):
        col = LU[k:, k]
        p = k + int(np.argmax(np.abs(col.real) + np.abs(col.imag)))
        piv[k] = p
        if LU[p, k] == 0:
            raise SingularMatrix(k + 1)
        if p != k:
            LU[[k, p], :] = LU[[p, k], :]
        LU[k + 1:, k] /= LU[k, k]
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
        yield k
    return LU, piv


def lu_factor(A: np.ndarray):
    """In-place style unblocked LU with partial pivoting: returns (LU, piv) with
    P A = L U, L unit lower (strictly below the diagonal of LU), piv[k] = row swapped with k."""
    g = lu_factor_columns(A)
    while True:
        try:
            next(g)
        except StopIteration as done:
            return done.value


def lu_solve(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B from lu_factor's output: row swaps, forward (unit L), backward (U)."""
    X = np.array(B, dtype=np.complex128, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = LU.shape[0]
    for k in range(n):
        p = piv[k]
        if p != k:
            X[[k, p], :] = X[[p, k], :]
    for i in range(1, n):
        X[i, :] -= LU[i, :i] @ X[:i, :]
    for i in range(n - 1, -1, -1):
        X[i, :] = (X[i, :] - LU[i, i + 1:] @ X[i + 1:, :]) / LU[i, i]
    return X[:, 0] if vec else X


def dense_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """x = A^{-1} b by the plain definition: full dense LU with partial pivoting."""
    LU, piv = lu_factor(A)
    return lu_solve(LU, piv, B)


def schur_complement(blocks) -> np.ndarray:
    """U33 = -M31 M13 - M32 M23 (Theorem thm:LU)."""
    M13, M23, M31, M32 = blocks
    return -(M31 @ M13) - (M32 @ M23)


def schur_solve(blocks, B: np.ndarray, factor=None) -> np.ndarray:
    """Solve the 3N mixed system for arbitrary 3N right-hand sides (Corollary lem:for_ssm_RHS)."""
    M13, M23, M31, M32 = blocks
    N = M13.shape[0]
    B = np.asarray(B, dtype=np.complex128)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    b1, b2, b3 = B[:N], B[N:2 * N], B[2 * N:]
    if factor is None:
        factor = lu_factor(schur_complement(blocks))
    LU, piv = factor
    z3 = lu_solve(LU, piv, b3 - M31 @ b1 - M32 @ b2)
    X = np.concatenate([b1 - M13 @ z3, b2 - M23 @ z3, z3], 0)
    return X[:, 0] if vec else X


def block_rhs_solve(blocks, B1: np.ndarray, B2: np.ndarray, B3: np.ndarray, factor=None) -> np.ndarray:
    """Solution for the block-diagonal right-hand side diag(B1, B2, B3), Corollary lem:block_LU:
    Z31 = -U33^{-1} M31 B1, Z32 = -U33^{-1} M32 B2, Z33 = U33^{-1} B3, then
    X = [[B1 - M13 Z31, -M13 Z32, -M13 Z33], [-M23 Z31, B2 - M23 Z32, -M23 Z33], [Z31, Z32, Z33]]."""
    M13, M23, M31, M32 = blocks
    N = M13.shape[0]
    B1, B2, B3 = (np.zeros((N, 0), np.complex128) if B is None else np.asarray(B, np.complex128).reshape(N, -1)
                  for B in (B1, B2, B3))
    if factor is None:
        factor = lu_factor(schur_complement(blocks))
    LU, piv = factor
    Z31 = -lu_solve(LU, piv, M31 @ B1)
    Z32 = -lu_solve(LU, piv, M32 @ B2)
    Z33 = lu_solve(LU, piv, B3)
    top = np.concatenate([B1 - M13 @ Z31, -M13 @ Z32, -M13 @ Z33], 1)
    mid = np.concatenate([-M23 @ Z31, B2 - M23 @ Z32, -M23 @ Z33], 1)
    bot = np.concatenate([Z31, Z32, Z33], 1)
    return np.concatenate([top, mid, bot], 0)


def mixed_residual(blocks, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """r = b - A x using the block structure of Eq. dis_mixedBM (identity/zero blocks not stored)."""
    M13, M23, M31, M32 = blocks
    N = M13.shape[0]
    x1, x2, x3 = X[:N], X[N:2 * N], X[2 * N:]
    b1, b2, b3 = B[:N], B[N:2 * N], B[2 * N:]
    return np.concatenate([b1 - x1 - M13 @ x3, b2 - x2 - M23 @ x3, b3 - M31 @ x1 - M32 @ x2], 0)


def mixed_norm_inf(blocks) -> float:
    """||A||_inf of the 3N mixed matrix (identity rows included)."""
    M13, M23, M31, M32 = blocks
    r1 = 1.0 + np.abs(M13).sum(1)
    r2 = 1.0 + np.abs(M23).sum(1)
    r3 = np.abs(M31).sum(1) + np.abs(M32).sum(1)
    return float(max(r1.max(), r2.max(), r3.max()))


def _eta(R, X, B, normA):
    R = R.reshape(R.shape[0], -1)
    X = X.reshape(X.shape[0], -1)
    B = B.reshape(B.shape[0], -1)
    num = np.abs(R).max(0)
    den = normA * np.abs(X).max(0) + np.abs(B).max(0)
    return float((num / den).max())


def backward_error_mixed(blocks, X, B) -> float:
    return _eta(mixed_residual(blocks, X, B), X, B, mixed_norm_inf(blocks))


def backward_error_dense(A, X, B) -> float:
    return _eta(B - A @ X, X, B, float(np.abs(A).sum(1).max()))

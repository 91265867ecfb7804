"""Pins for the oracle's dense linear algebra: LAPACK (numpy.linalg.solve) for the unblocked LU,
the full 3N dense LU for the Schur path of Theorem thm:LU / Corollary lem:for_ssm_RHS."""
import numpy as np
import pytest

import workloads as W
import oracle as O
from oracle.dense import SingularMatrix, lu_factor, lu_solve, schur_solve, schur_complement


def _rand(n, m=None, seed=0):
    rng = np.random.default_rng(seed)
    m = n if m is None else m
    return rng.normal(size=(n, m)) + 1j * rng.normal(size=(n, m))


def test_lu_matches_lapack():
    A = _rand(97, seed=1)
    B = _rand(97, 5, seed=2)
    X = lu_solve(*lu_factor(A), B)
    Xr = np.linalg.solve(A, B)
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) < 1e-12


def test_lu_reconstructs_PA_eq_LU_and_bounds_L():
    A = _rand(40, seed=3)
    LU, piv = lu_factor(A)
    L = np.tril(LU, -1) + np.eye(40)
    U = np.triu(LU)
    PA = A.copy()
    for k, p in enumerate(piv):
        PA[[k, p]] = PA[[p, k]]
    assert np.abs(PA - L @ U).max() < 1e-12
    assert (np.abs(L.real) + np.abs(L.imag)).max() <= 2.0 + 1e-12    # |l| <= 1 in the pivot norm


def test_pivot_tie_break_first_index():
    A = np.array([[1.0, 2.0], [1.0, 3.0]], dtype=complex)            # tie in column 0
    _, piv = lu_factor(A)
    assert piv[0] == 0


def test_singular_reports_column():
    A = _rand(6, seed=4)
    A[:, 2] = 0.0                      # stays exactly zero through elimination -> 1-based column 3
    with pytest.raises(SingularMatrix) as e:
        lu_factor(A)
    assert e.value.col == 3


def test_schur_path_equals_dense_3N_random_rhs():
    g = O.nodes(W.ellipse(1.0, 0.6), 48)
    P = O.default_params(2.0, 3.0)
    blocks = O.mixed_blocks(g, P)
    A = O.mixed_matrix(blocks)
    B = W.gaussian_full(3 * 48, 4, seed=7)                           # b1, b2 != 0: Corollary case
    X = schur_solve(blocks, B)
    Xr = np.linalg.solve(A, B)
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) < 1e-12
    assert O.backward_error_mixed(blocks, X, B) < 1e-14


def test_theorem_factor_blocks():
    # U33 of Theorem thm:LU equals the trailing block of one step of block Gaussian elimination
    # of the full 3N matrix (eliminate the two identity blocks first).
    g = O.nodes(W.circle(1.0), 32)
    P = O.default_params(2.0, 3.0)
    M13, M23, M31, M32 = O.mixed_blocks(g, P)
    A = O.mixed_matrix((M13, M23, M31, M32))
    N = 32
    A11 = A[:2 * N, :2 * N]
    A12 = A[:2 * N, 2 * N:]
    A21 = A[2 * N:, :2 * N]
    S = A[2 * N:, 2 * N:] - A21 @ np.linalg.solve(A11, A12)
    assert np.abs(S - schur_complement((M13, M23, M31, M32))).max() < 1e-13


def test_backward_error_definition():
    A = _rand(30, seed=5)
    X = _rand(30, 2, seed=6)
    B = A @ X
    assert O.backward_error_dense(A, X, B) < 1e-15
    Xp = X.copy()
    Xp[0, 0] += 1e-6
    eta = O.backward_error_dense(A, Xp, B)
    assert 1e-9 < eta < 1e-6


def test_block_rhs_corollary_equals_dense_3N():
    # Corollary lem:block_LU against LAPACK on the full 3N matrix with the block-diagonal
    # right-hand side diag(B1, B2, B3) (widths 2, 3, 1), and with an empty block
    N = 40
    g = O.nodes(W.star(1.0, 0.25, 4), N)
    blocks = O.mixed_blocks(g, O.default_params(3.0 - 0.1j, 4.5))
    A = O.mixed_matrix(blocks)
    B1, B2, B3 = _rand(N, 2, seed=11), _rand(N, 3, seed=12), _rand(N, 1, seed=13)
    Bd = np.zeros((3 * N, 6), dtype=complex)
    Bd[:N, :2], Bd[N:2 * N, 2:5], Bd[2 * N:, 5:] = B1, B2, B3
    X = O.block_rhs_solve(blocks, B1, B2, B3)
    Xr = np.linalg.solve(A, Bd)
    assert X.shape == (3 * N, 6)
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) < 1e-12
    X2 = O.block_rhs_solve(blocks, None, B2, B3)
    assert np.linalg.norm(X2 - Xr[:, 2:]) / np.linalg.norm(Xr[:, 2:]) < 1e-12

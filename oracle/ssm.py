"""Oracle: block Sakurai-Sugiura projection (Hankel form) for the nonlinear eigenvalue problem
T(omega) x = 0 of the discretised boundary integral equations (test infrastructure only).

§5.3 (sec:ssm) uses the Sakurai-Sugiura projection method to find the complex omega for which the
discretised direct-indirect system (Eq. dis_mixedBM) or the ordinary system (Eq. dis_BM) is
singular, solving the system at quadrature points of a closed contour with random right-hand
sides (which is where Corollary lem:for_ssm_RHS - arbitrary 3N right-hand sides - comes in).  The
paper cites the method and gives its parameters (Table tb:ssm_parameters) but not its steps; this
module takes the block Hankel variant of that method:

  contour  circle of centre gamma and radius rho, P trapezoid points
           z_p = gamma + rho zeta_p, zeta_p = exp(i theta_p), theta_p = 2 pi (p + 1/2) / P
  weights  (1 / 2 pi i) oint f dz ~ sum_p w_p f(z_p), w_p = rho zeta_p / P
  moments  mu_k = sum_p w_p zeta_p^k U^H T(z_p)^{-1} V, k = 0 .. 2M - 1 (L x L each; V, U: n x L)
  Hankel   H = [mu_{i+j}], Hs = [mu_{i+j+1}], i, j = 0 .. M - 1 (LM x LM)
  rank     H = W1 S W2^H, r = #{s_i > delta s_1}
  pencil   B = W1_r^H Hs W2_r S_r^{-1}; its eigenvalues zeta give omega = gamma + rho zeta,
           kept when |zeta| < 1 (inside the contour).

Library routines serve as steps: the dense solves (numpy), the SVD and the small eigenproblem.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from .geometry import nodes
from .systems import default_params, mixed_blocks, mixed_matrix, ordinary_matrix


def contour(center: complex, radius: float, P: int):
    """Trapezoid points z_p, normalised points zeta_p and weights w_p on a circle."""
    theta = 2.0 * np.pi * (np.arange(P) + 0.5) / P
    zeta = np.exp(1j * theta)
    return center + radius * zeta, zeta, radius * zeta / P


def moments(solve, center: complex, radius: float, P: int, M: int, V: np.ndarray, U: np.ndarray | None = None):
    """mu_k, k = 0 .. 2M-1, for a callable solve(z, V) = T(z)^{-1} V."""
    U = V if U is None else U
    z, zeta, w = contour(center, radius, P)
    L = V.shape[1]
    mu = np.zeros((2 * M, L, L), dtype=np.complex128)
    for p in range(P):
        Pp = U.conj().T @ solve(z[p], V)
        for k in range(2 * M):
            mu[k] += w[p] * zeta[p] ** k * Pp
    return mu


def hankel_eigs(mu: np.ndarray, center: complex, radius: float, delta: float = 1e-12):
    """Eigenvalues inside the contour from the moments; returns (omega_inside, all_omega, singular values)."""
    twoM, L, _ = mu.shape
    M = twoM // 2
    H = np.zeros((L * M, L * M), dtype=np.complex128)
    Hs = np.zeros_like(H)
    for i in range(M):
        for j in range(M):
            H[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j]
            Hs[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j + 1]
    W1, s, W2h = np.linalg.svd(H)
    r = int(np.sum(s > delta * s[0]))
    B = W1[:, :r].conj().T @ Hs @ W2h[:r].conj().T @ np.diag(1.0 / s[:r])
    zeta = np.linalg.eigvals(B)
    omega = center + radius * zeta
    inside = omega[np.abs(zeta) < 1.0]
    return np.sort_complex(inside), omega, s


def bie_solver(curve: W.Curve, N: int, k_ratio: complex, formulation: int, zeta_p: int = 0):
    """solve(z, V) = T(z)^{-1} V for the discretised system at k_out = z, k_in = k_ratio z (so
    eps1 = k_ratio^2 is fixed along the contour; beta = i / k_out).  zeta_p > 0 assembles with the
    high-order zeta-corrected rule of §5.3 (order 2 zeta_p + 3, ``oracle.zeta``)."""
    g = nodes(curve, N)

    def solve(z, V):
        P = default_params(z, k_ratio * z)
        if formulation == W.MIXED:
            A = mixed_matrix(mixed_blocks(g, P, zeta_p))
        else:
            A = ordinary_matrix(g, P, zeta_p=zeta_p)
        return np.linalg.solve(A, V)

    return solve


def ssm(curve: W.Curve, N: int, k_ratio: complex, formulation: int, center: complex, radius: float, P: int, M: int,
        V: np.ndarray, delta: float = 1e-12, zeta_p: int = 0):
    """Eigenvalues of the discretised system inside the circle (block Hankel Sakurai-Sugiura)."""
    mu = moments(bie_solver(curve, N, k_ratio, formulation, zeta_p), center, radius, P, M, V)
    return hankel_eigs(mu, center, radius, delta)

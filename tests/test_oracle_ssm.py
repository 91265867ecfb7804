"""Pins for the oracle's block Sakurai-Sugiura solver (oracle/ssm.py, §5.3 sec:ssm).

* A linear problem T(z) = A - z I with known eigenvalues: exactly those inside the circle come
  back (to 1e-10), whatever lies outside - a wrong weight, a shifted moment index or a transposed
  Hankel block breaks this.
* The paper's own check (Table tb:ssm_eigenvalues, setting of Table tb:ssm_parameters: circle of
  radius 0.5, eps1 = 4, so the eigen-relation H_n(k1 a) = 0 puts eigenvalues at the zeros of
  H_n^(1)(omega)): both formulations find the double eigenvalue (n = +-2) at the tabulated zero of
  H_2^(1), and n = 3 at H_3^(1), with the third-order convergence of the quadrature
  (error / 8 per doubling of N).
"""
import os

import numpy as np

import workloads as W
from oracle import ssm

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hankel_zeros.txt")


def _zero(n):
    for line in open(GOLD):
        f = line.split()
        if f and f[0] == str(n) and f[1] == "reference_doring":
            return complex(float(f[2]), float(f[3]))
    raise KeyError(n)


def test_linear_problem_exact_eigenvalues():
    rng = np.random.default_rng(0)
    n = 40
    lam = np.array([0.3 + 0.1j, -0.2 - 0.25j, 0.1 + 0.05j, 0.9 + 0.9j, 2.0, -1.5j] + list(3 + rng.normal(size=34)))
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    V = rng.normal(size=(n, 4)) + 1j * rng.normal(size=(n, 4))
    mu = ssm.moments(lambda z, B: np.linalg.solve(A - z * np.eye(n), B), 0.0, 0.5, 32, 4, V)
    inside, _, s = ssm.hankel_eigs(mu, 0.0, 0.5, 1e-12)
    ref = np.sort_complex(lam[np.abs(lam) < 0.5])
    assert inside.size == ref.size == 3
    assert np.abs(inside - ref).max() < 1e-10


def test_contour_quadrature_weights():
    # (1/2 pi i) oint z^k dz = 0 for k >= 0, (1/2 pi i) oint dz / z = 1 on a circle around 0
    z, zeta, w = ssm.contour(0.3 - 0.2j, 0.7, 16)
    assert abs(np.sum(w / (z - (0.3 - 0.2j))) - 1.0) < 1e-14
    assert abs(np.sum(w * z ** 3)) < 1e-13


def test_hankel_zero_eigenvalues_both_formulations():
    target = _zero(2)
    errs = []
    for N in (64, 128):
        V = W.gaussian_full(3 * N, 4, 3)
        inside, _, _ = ssm.ssm(W.circle(0.5), N, 2.0, W.MIXED, target, 0.05, 32, 4, V)
        assert inside.size == 2                        # n = +2 and n = -2
        errs.append(np.abs(inside - target).max())
    assert errs[1] < 5e-6 and errs[0] / errs[1] > 6.0   # O(h^3): ~8 per doubling
    V = W.gaussian_full(2 * 128, 4, 3)
    inside, _, _ = ssm.ssm(W.circle(0.5), 128, 2.0, W.ORDINARY, target, 0.05, 32, 4, V)
    assert inside.size == 2 and np.abs(inside - target).max() < 5e-6


def test_hankel_zero_n3():
    target = _zero(3)
    V = W.gaussian_full(3 * 128, 4, 4)
    inside, _, _ = ssm.ssm(W.circle(0.5), 128, 2.0, W.MIXED, target, 0.05, 32, 4, V)
    assert inside.size == 2 and np.abs(inside - target).max() < 5e-5

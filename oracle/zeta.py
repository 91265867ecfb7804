"""High-order zeta-corrected trapezoidal rule for the layer operators (test infrastructure only).

§4 discretises S_k, D_k, D*_k and N_k with the zeta-corrected trapezoidal rule [wu2023unified]
with one local correction point; §5.3 uses a high-order version of the same rule ("order 31")
for the contour eigenvalue computation.  The correction weights are not printed; this module
derives them from the generalised Euler-Maclaurin expansion of the punctured trapezoidal sum
(Navot), which is what the zeta correction is built on:

    for smooth g and the equispaced nodes x_j = j h,
    int |x|^s g(x) dx = h sum_{j != 0} |jh|^s g(jh) - 2 sum_{k >= 0} zeta(-s-2k) h^(s+2k+1) g^(2k)(0) / (2k)!

(the integral over a neighbourhood of the singular node; the far part of a periodic integrand
is integrated spectrally by the plain sum).  Two cases occur in the 2-D kernels:

* log|x| (the s-derivative at s = 0; zeta(-2k) = 0 for k >= 1):
      correction = h ln(h / 2pi) g(0) + 2 sum_{k>=1} zeta'(-2k) h^(2k+1) g^(2k)(0) / (2k)!.
  Replacing the derivatives by the symmetric stencil g(mh), |m| <= p, exact for even
  polynomials of degree <= 2p, gives weights h tau_m with
      sum_{m=1..p} tau_m m^(2k) = zeta'(-2k)   (k = 1..p),   tau_0 = ln(h/2pi) - 2 sum_{m>=1} tau_m,
  and an O(h^(2p+3)) rule.  zeta'(-2k) = (-1)^k (2k)! zeta(2k+1) / (2 (2pi)^(2k)) by the
  functional equation.
* x^-2 (Hadamard finite part; zeta(0) = -1/2 and zeta(-2k) = 0 for k >= 1, so the expansion
  stops after two terms):
      correction = -(pi^2 / 3h) g(0) + (h / 2) g''(0),
  with g''(0) from the central stencil over |m| <= p + 1 (error O(h^(2p+2))), so this part is
  O(h^(2p+3)) as well.

Kernel splitting (row i = target t, column j = source s, x = s - t, d = x(t) - x(s)): the
logarithmic parts come from the log(z/2) J_n(z) terms of Y_0 and Y_1, with log r = log|x| +
log(r/|x|) and r/|x| smooth and positive:
    A_S  = -(1/2pi) J0(kr)                                             |x'(s)|
    A_D  = -(k/2pi) J1(kr) (d.nu_s)/r                                  |x'(s)|
    A_D* = +(k/2pi) J1(kr) (d.nu_t)/r                                  |x'(s)|
    A_N  = -(k/2pi) [k J0 (d.nu_t)(d.nu_s)/r^2 - 2 J1 (d.nu_t)(d.nu_s)/r^3 + J1 (nu_t.nu_s)/r] |x'(s)|
and N's remaining part behaves as a_{-2}/x^2 + a_{-1}/x + smooth with a_{-2} = 1/(2pi |x'(t)|)
(the odd term needs no correction on a symmetric stencil).  At s = t: A_S -> -|x'|/2pi,
A_D = A_D* -> 0, A_N -> -(k^2/4pi) |x'|.

p = 0 is the paper's one-point rule (the oracle's layer_operators): tau_0 = ln(h/2pi) on the
diagonal and no finite-difference term for N, whose rule is then O(h).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
from scipy import special as sp

from .geometry import Geometry


def zeta_prime_at_negative_even(k: int) -> float:
    """zeta'(-2k) for k >= 1, from zeta(2k+1) by the functional equation."""
    return (-1) ** k * math.factorial(2 * k) * float(sp.zeta(2 * k + 1, 1)) / (2.0 * (2.0 * math.pi) ** (2 * k))


def _solve_exact(A, b):
    """Gauss-Jordan elimination in exact rationals (small dense systems)."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [v / pv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [v - f * w for v, w in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


@lru_cache(maxsize=None)
def log_weights(p: int) -> tuple:
    """tau_1..tau_p of the log-singular correction (the m = 0 weight is ln(h/2pi) - 2 sum)."""
    if p <= 0:
        return ()
    A = [[Fraction(m ** (2 * k)) for m in range(1, p + 1)] for k in range(1, p + 1)]
    b = [Fraction(zeta_prime_at_negative_even(k)) for k in range(1, p + 1)]
    return tuple(float(v) for v in _solve_exact(A, b))


@lru_cache(maxsize=None)
def second_derivative_weights(q: int) -> tuple:
    """c_0..c_q of the central stencil g''(0) ~ h^-2 sum_{|m|<=q} c_|m| g(mh), exact for
    polynomials of degree <= 2q + 1."""
    A = [[Fraction(1 if k == 0 else 0)] + [Fraction(2 * m ** (2 * k)) for m in range(1, q + 1)]
         for k in range(q + 1)]
    b = [Fraction(2 if k == 1 else 0) for k in range(q + 1)]
    return tuple(float(v) for v in _solve_exact(A, b))


def log_coefficients(g: Geometry, k: complex, I: np.ndarray, J: np.ndarray) -> dict:
    """A_S, A_D, A_D*, A_N times the trapezoid weight w_j, at pairs (I, J) with I != J."""
    d = g.x[I] - g.x[J]
    r = np.hypot(d[..., 0], d[..., 1])
    dni = d[..., 0] * g.nu[I, 0] + d[..., 1] * g.nu[I, 1]
    dnj = d[..., 0] * g.nu[J, 0] + d[..., 1] * g.nu[J, 1]
    ninj = g.nu[I, 0] * g.nu[J, 0] + g.nu[I, 1] * g.nu[J, 1]
    z = complex(k) * r
    J0, J1 = sp.jv(0, z), sp.jv(1, z)
    wj = g.w[J]
    c = complex(k) / (2 * np.pi)
    return {
        "S": -J0 / (2 * np.pi) * wj,
        "D": -c * J1 * dnj / r * wj,
        "Ds": c * J1 * dni / r * wj,
        "N": -c * (complex(k) * J0 * dni * dnj / r ** 2 - 2.0 * J1 * dni * dnj / r ** 3 + J1 * ninj / r) * wj,
    }


def apply_corrections(g: Geometry, k: complex, ops: dict, p: int) -> dict:
    """The order-(2p+3) rule from the one-point matrices ``ops`` (keys S, D, Ds, N; modified
    copies are returned): log-term weights on the 2p+1 nodes around each diagonal, and for N
    the second-derivative term of the x^-2 part on 2p+3 nodes."""
    if p <= 0:
        return ops
    N = g.N
    if 2 * (p + 1) + 1 > N:
        raise ValueError(f"{N} nodes cannot carry a correction stencil of {p} points")
    out = {key: A.copy() for key, A in ops.items()}
    h = g.h
    tau = log_weights(p)
    c2 = second_derivative_weights(p + 1)
    rows = np.arange(N)
    # diagonal: the m = 0 log weight beyond ln(h/2pi), and N's stencil centre
    sig0 = -2.0 * sum(tau)
    out["S"][rows, rows] += sig0 * (-g.w / (2 * np.pi))
    out["N"][rows, rows] += sig0 * (-(complex(k) ** 2) / (4 * np.pi) * g.w)
    out["N"][rows, rows] += c2[0] * (1.0 / (2 * np.pi * g.speed)) / (2 * h)
    for m in range(1, p + 2):
        for sgn in (1, -1):
            cols = (rows + sgn * m) % N
            A = log_coefficients(g, k, rows, cols)
            if m <= p:
                for key in ("S", "D", "Ds", "N"):
                    out[key][rows, cols] += tau[m - 1] * A[key]
            # N: x^2 times the non-log part, from the one-point (plain trapezoid) entries
            nonlog = ops["N"][rows, cols] - A["N"] * np.log(m * h)
            out["N"][rows, cols] += 0.5 * c2[m] * m * m * nonlog
    return out

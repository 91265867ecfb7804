"""Oracle boundary integral operators S_k, D_k, D*_k, N_k (test infrastructure only).

Kernels (§2.2): G(x, y; k) = (i/4) H0^(1)(k|x - y|), d = 2.  With d = x_i - y_j,
r = |d|, nu_i = nu(x_i), nu_j = nu(y_j), and H0' = -H1, the normal derivatives give,
for i != j (row i = target, column j = source, weight w_j = h |x'(t_j)|):

    S[i,j]  = (i/4)  H0(kr)                                  w_j
    D[i,j]  = (ik/4) H1(kr) (d.nu_j)/r                       w_j      dG/dnu(y)
    D*[i,j] = -(ik/4) H1(kr) (d.nu_i)/r                      w_j      dG/dnu(x)
    N[i,j]  = (ik/4)[ k H0 (d.nu_i)(d.nu_j)/r^2
                      - 2 H1 (d.nu_i)(d.nu_j)/r^3 + H1 (nu_i.nu_j)/r ] w_j

Diagonal (§4: zeta-corrected trapezoid rule with one local correction point,
read as "correct the leading singular term at i = j only"):

* S: the log singularity -(1/4pi) ln(4 sin^2((t-s)/2)) |x'| has the one-point
  weight 2h ln(h/2pi); the smooth remainder at t = s is
  i/4 - (1/2pi)(ln(k/2) + gamma) - (1/2pi) ln|x'|.  Together
  S[i,i] = w_i [ i/4 - (ln(k/2) + gamma)/(2pi) - ln(w_i / 2pi)/(2pi) ].
* D, D*: smooth limit of the kernel, -kappa_i/(4pi), times w_i.
* N: the (t-s)^-2 singularity with coefficient 1/(2pi |x'_i|) gets the
  zeta weight -pi^2/(3h); the -(k^2/4pi) ln r singularity gets the log weight;
  the O(h) smooth remainder is dropped (the paper states O(h) for N_k):
  N[i,i] = -pi/(6 h |x'_i|) - (k^2/4pi) ln(h/2pi) w_i.

Hankel functions come from scipy.special (AMOS), a library primitive
independent of the CUDA implementation; tests pin it to mpmath.
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp

from .geometry import Geometry

EULER_GAMMA = 0.57721566490153286060651209008240243


def hankel01(z):
    """H0^(1)(z), H1^(1)(z) for complex z (principal branch), via scipy.special.hankel1."""
    z = np.asarray(z, dtype=np.complex128)
    return sp.hankel1(0, z), sp.hankel1(1, z)


def _offdiag(g: Geometry, k: complex, I: np.ndarray, J: np.ndarray):
    """Kernel values for index pairs (I, J) with I != J; returns S, D, D*, N entries."""
    d = g.x[I] - g.x[J]
    r = np.hypot(d[..., 0], d[..., 1])
    dni = d[..., 0] * g.nu[I, 0] + d[..., 1] * g.nu[I, 1]
    dnj = d[..., 0] * g.nu[J, 0] + d[..., 1] * g.nu[J, 1]
    ninj = g.nu[I, 0] * g.nu[J, 0] + g.nu[I, 1] * g.nu[J, 1]
    H0, H1 = hankel01(k * r)
    wj = g.w[J]
    S = 0.25j * H0 * wj
    D = 0.25j * k * H1 * dnj / r * wj
    Ds = -0.25j * k * H1 * dni / r * wj
    Nk = 0.25j * k * (k * H0 * dni * dnj / r ** 2 - 2.0 * H1 * dni * dnj / r ** 3 + H1 * ninj / r) * wj
    return S, D, Ds, Nk


def _diag(g: Geometry, k: complex, I: np.ndarray):
    """Zeta-corrected diagonal entries (one local correction point) for rows I."""
    k = complex(k)
    w = g.w[I]
    S = w * (0.25j - (np.log(k / 2.0) + EULER_GAMMA) / (2 * np.pi) - np.log(w / (2 * np.pi)) / (2 * np.pi))
    D = -g.kappa[I] * w / (4 * np.pi) + 0j
    Ds = D.copy()
    Nk = -np.pi / (6.0 * g.h * g.speed[I]) - (k * k / (4 * np.pi)) * np.log(g.h / (2 * np.pi)) * w
    return S, D, Ds, Nk + 0j


def layer_operators(g: Geometry, k: complex, zeta_p: int = 0) -> dict:
    """Full N x N matrices S_k, D_k, D*_k, N_k (keys 'S', 'D', 'Ds', 'N').  zeta_p > 0 adds the
    order-(2 zeta_p + 3) zeta corrections of ``oracle.zeta`` (the §5.3 high-order rule)."""
    N = g.N
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    off = I != J
    out = {key: np.zeros((N, N), dtype=np.complex128) for key in ("S", "D", "Ds", "N")}
    vals = _offdiag(g, k, I[off], J[off])
    for key, v in zip(("S", "D", "Ds", "N"), vals):
        out[key][off] = v
    dvals = _diag(g, k, np.arange(N))
    for key, v in zip(("S", "D", "Ds", "N"), dvals):
        out[key][np.arange(N), np.arange(N)] = v
    if zeta_p > 0:
        from .zeta import apply_corrections
        out = apply_corrections(g, k, out, zeta_p)
    return out


def layer_entries(g: Geometry, k: complex, I, J) -> dict:
    """Operator entries at arbitrary index pairs (I, J) (diagonal pairs allowed)."""
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    out = {key: np.zeros(I.shape, dtype=np.complex128) for key in ("S", "D", "Ds", "N")}
    off = I != J
    if off.any():
        for key, v in zip(("S", "D", "Ds", "N"), _offdiag(g, k, I[off], J[off])):
            out[key][off] = v
    on = ~off
    if on.any():
        for key, v in zip(("S", "D", "Ds", "N"), _diag(g, k, I[on])):
            out[key][on] = v
    return out

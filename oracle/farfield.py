"""Oracle far-field pattern from boundary data (test infrastructure only).

Not printed in the paper; derived from the exterior Green representation used
for the Burton-Miller equation of §3.1 (total field u on Gamma, du/dnu = eps0 q)
and the large-argument form of G = (i/4) H0^(1):

    u_inf(xhat) = e^{i pi/4} / sqrt(8 pi k0) * int_Gamma [ -i k0 (xhat.nu) u - eps0 q ] e^{-i k0 xhat.y} ds(y)

evaluated with the trapezoid weights w_j = h |x'(t_j)|.
"""
from __future__ import annotations

import numpy as np

from .geometry import Geometry


def far_field(g: Geometry, k0: complex, eps0: complex, u: np.ndarray, q: np.ndarray, angles) -> np.ndarray:
    """u_inf at the given observation angles; u, q are (N,) or (N, nrhs)."""
    angles = np.asarray(angles, dtype=np.float64)
    xh = np.stack([np.cos(angles), np.sin(angles)], 1)           # (M, 2)
    ph = np.exp(-1j * k0 * (xh @ g.x.T))                          # (M, N)
    xn = xh @ g.nu.T                                              # (M, N)
    c = np.exp(0.25j * np.pi) / np.sqrt(8.0 * np.pi * k0)
    u2 = u if u.ndim == 2 else u[:, None]
    q2 = q if q.ndim == 2 else q[:, None]
    F = c * (((-1j * k0) * xn * ph * g.w[None, :]) @ u2 - eps0 * (ph * g.w[None, :]) @ q2)
    return F if u.ndim == 2 else F[:, 0]

"""Oracle geometry: equispaced Nystrom nodes on a closed curve (test infrastructure only).

§4 (discretisation): N quadrature points equally spaced in the curve parameter
t in [0, 2*pi), h = 2*pi/N, t_j = j h.  §2.1: the unit normal points into the
exterior Omega_0; with a counter-clockwise parametrisation that is
nu = (y', -x') / |x'|.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

import workloads as W


@dataclass
class Geometry:
    N: int
    h: float
    t: np.ndarray        # (N,)
    x: np.ndarray        # (N, 2) nodes
    dx: np.ndarray       # (N, 2) x'(t)
    ddx: np.ndarray      # (N, 2) x''(t)
    speed: np.ndarray    # |x'(t)|
    nu: np.ndarray       # (N, 2) outward unit normal
    kappa: np.ndarray    # signed curvature (x'y'' - y'x'')/|x'|^3
    w: np.ndarray        # trapezoid weights h |x'(t_j)|


def _curve_derivs(curve: W.Curve, t: np.ndarray):
    p = curve.params4()
    c, s = np.cos(t), np.sin(t)
    if curve.kind == W.CIRCLE:
        R, cx, cy = p[0], p[1], p[2]
        x = np.stack([cx + R * c, cy + R * s], 1)
        dx = np.stack([-R * s, R * c], 1)
        ddx = np.stack([-R * c, -R * s], 1)
    elif curve.kind == W.ELLIPSE:
        a, b = p[0], p[1]
        x = np.stack([a * c, b * s], 1)
        dx = np.stack([-a * s, b * c], 1)
        ddx = np.stack([-a * c, -b * s], 1)
    elif curve.kind == W.STAR:
        r0, amp, m = p[0], p[1], p[2]
        r = r0 + amp * np.cos(m * t)
        dr = -amp * m * np.sin(m * t)
        ddr = -amp * m * m * np.cos(m * t)
        x = np.stack([r * c, r * s], 1)
        dx = np.stack([dr * c - r * s, dr * s + r * c], 1)
        ddx = np.stack([ddr * c - 2 * dr * s - r * c, ddr * s + 2 * dr * c - r * s], 1)
    elif curve.kind == W.KITE:
        cc, b = p[0], p[1]
        x = np.stack([c + cc * np.cos(2 * t) - cc, b * s], 1)
        dx = np.stack([-s - 2 * cc * np.sin(2 * t), b * c], 1)
        ddx = np.stack([-c - 4 * cc * np.cos(2 * t), -b * s], 1)
    else:
        raise ValueError(f"curve kind {curve.kind} has no analytic form in the oracle")
    return x, dx, ddx


def nodes(curve: W.Curve, N: int) -> Geometry:
    """Nodes, tangents, normals, curvature and trapezoid weights at t_j = 2*pi*j/N."""
    if N < 3:
        raise ValueError("need N >= 3 nodes")
    h = 2.0 * np.pi / N
    t = h * np.arange(N)
    x, dx, ddx = _curve_derivs(curve, t)
    speed = np.hypot(dx[:, 0], dx[:, 1])
    nu = np.stack([dx[:, 1], -dx[:, 0]], 1) / speed[:, None]
    kappa = (dx[:, 0] * ddx[:, 1] - dx[:, 1] * ddx[:, 0]) / speed ** 3
    return Geometry(N, h, t, x, dx, ddx, speed, nu, kappa, h * speed)

"""Pins for the oracle's node geometry: closed-form perimeters/areas, Gauss-Bonnet, orientation."""
import numpy as np
from scipy import special as sp

import workloads as W
from oracle import nodes


def test_circle_exact():
    g = nodes(W.circle(0.7, 0.1, -0.2), 50)
    c = np.array([0.1, -0.2])
    assert np.allclose(np.hypot(*(g.x - c).T), 0.7, atol=1e-15)
    assert np.allclose(g.kappa, 1 / 0.7, rtol=1e-14)
    assert np.allclose(g.nu, (g.x - c) / 0.7, atol=1e-14)      # outward
    assert abs(g.w.sum() - 2 * np.pi * 0.7) < 1e-13


def test_ellipse_perimeter_and_curvature():
    a, b = 1.0, 0.6
    g = nodes(W.ellipse(a, b), 256)
    perim = 4 * a * sp.ellipe(1 - (b / a) ** 2)
    assert abs(g.w.sum() - perim) < 1e-12
    assert abs(g.kappa[0] - a / b ** 2) < 1e-12                 # vertex curvature a/b^2
    assert abs(g.kappa[g.N // 4] - b / a ** 2) < 1e-12


def _area(g):
    # (1/2) \oint (x dy - y dx) with the trapezoid rule (spectral for periodic data)
    return 0.5 * g.h * np.sum(g.x[:, 0] * g.dx[:, 1] - g.x[:, 1] * g.dx[:, 0])


def test_star_and_kite_area_gauss_bonnet():
    gs = nodes(W.star(1.0, 0.3, 5), 512)
    assert abs(_area(gs) - np.pi * (1.0 + 0.3 ** 2 / 2)) < 1e-12
    gk = nodes(W.kite(0.65, 1.5), 512)
    assert abs(_area(gk) - np.pi * 1.5) < 1e-12
    for g in (gs, gk, nodes(W.ellipse(), 300)):
        assert abs(np.sum(g.kappa * g.w) - 2 * np.pi) < 1e-10      # total curvature 2 pi
        assert np.abs(g.w @ g.nu).max() < 1e-12                    # \oint nu ds = 0
        assert np.allclose(np.hypot(*g.nu.T), 1.0)
        assert np.allclose(np.sum(g.nu * g.dx, 1), 0.0, atol=1e-13)  # normal is orthogonal to tangent

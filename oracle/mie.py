"""Oracle Bessel-series (Mie) solution for a circular transmissive scatterer (test infrastructure only).

§5.1 compares against the analytical solution on a circle without printing it;
it follows from the transmission problem (Eq. problem, §2.1) on a circle of
radius a centred at the origin, incident plane wave u_in = exp(i k0 x1):

    u_in  = sum_m i^m J_m(k0 r) e^{im theta}             (Jacobi-Anger)
    u0_sc = sum_m a_m H_m(k0 r) e^{im theta},   u1_sc = sum_m b_m J_m(k1 r) e^{im theta}

and the two transmission conditions at r = a (u continuous, (1/eps) du/dr continuous):

    i^m J_m(k0 a) + a_m H_m(k0 a) = b_m J_m(k1 a)
    (k0/eps0)[i^m J_m'(k0 a) + a_m H_m'(k0 a)] = (k1/eps1) b_m J_m'(k1 a)

The determinant of this 2x2 system is, up to sign and the factor 1/(eps0 eps1),
the first circle eigen-relation printed in §5.3.  Boundary data:
u = sum b_m J_m(k1 a) e^{im theta}, q = (k1/eps1) sum b_m J_m'(k1 a) e^{im theta}.
Far field (u_sc ~ e^{ik0 r} r^{-1/2} u_inf):
u_inf(theta) = sqrt(2/(pi k0)) e^{-i pi/4} sum_m a_m (-i)^m e^{im theta}.
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def mie_coefficients(a, k0, k1, eps0, eps1, mmax=None):
    """(m, a_m, b_m) for |m| <= mmax (default |k1| a + 40)."""
    if mmax is None:
        mmax = int(abs(k1) * a + 40)
    m = np.arange(-mmax, mmax + 1)
    z0, z1 = k0 * a, k1 * a
    J0, dJ0 = sp.jv(m, z0), sp.jvp(m, z0)
    H0, dH0 = sp.hankel1(m, z0), sp.h1vp(m, z0)
    J1, dJ1 = sp.jv(m, z1), sp.jvp(m, z1)
    im = (1j) ** m
    # [ H0          -J1            ] [a]   [ -im J0          ]
    # [ k0/e0 dH0   -k1/e1 dJ1     ] [b] = [ -k0/e0 im dJ0   ]
    A11, A12 = H0, -J1
    A21, A22 = (k0 / eps0) * dH0, -(k1 / eps1) * dJ1
    r1, r2 = -im * J0, -(k0 / eps0) * im * dJ0
    det = A11 * A22 - A12 * A21
    am = (r1 * A22 - A12 * r2) / det
    bm = (A11 * r2 - r1 * A21) / det
    return m, am, bm


def mie_boundary(a, k0, k1, eps0, eps1, theta):
    """Analytical u and q at boundary angles theta (circle radius a)."""
    m, am, bm = mie_coefficients(a, k0, k1, eps0, eps1)
    E = np.exp(1j * np.outer(theta, m))
    u = E @ (bm * sp.jv(m, k1 * a))
    q = E @ ((k1 / eps1) * bm * sp.jvp(m, k1 * a))
    return u, q


def mie_far_field(a, k0, k1, eps0, eps1, theta):
    m, am, bm = mie_coefficients(a, k0, k1, eps0, eps1)
    E = np.exp(1j * np.outer(theta, m))
    return np.sqrt(2.0 / (np.pi * k0)) * np.exp(-0.25j * np.pi) * (E @ (am * (-1j) ** m))

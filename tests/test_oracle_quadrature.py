"""Pins for the oracle's zeta-corrected Nystrom operators: on a circle every operator matrix is
circulant and its eigenvalues converge to closed forms obtained from Graf's addition theorem:

    S_m  = (i pi a / 2) J_m(ka) H_m(ka)
    D_m  = D*_m = (i pi k a / 4) (J_m'(ka) H_m(ka) + J_m(ka) H_m'(ka))
    N_m  = (i pi k^2 a / 2) J_m'(ka) H_m'(ka)

§4 states at least O(h^2) for S, D, D* and at least O(h) for N with the one-point correction.
A wrong diagonal constant (a dropped ln(k/2), gamma or curvature term, a wrong sign or factor)
leaves an O(h) error in S/D and fails the rate check; a wrong hypersingular weight leaves O(1)."""
import numpy as np
import pytest
from scipy import special as sp

import workloads as W
from oracle import nodes, layer_operators


def _closed(a, k, m):
    z = k * a
    J, dJ = sp.jv(m, z), sp.jvp(m, z)
    H, dH = sp.hankel1(m, z), sp.h1vp(m, z)
    return {
        "S": 0.5j * np.pi * a * J * H,
        "D": 0.25j * np.pi * k * a * (dJ * H + J * dH),
        "Ds": 0.25j * np.pi * k * a * (dJ * H + J * dH),
        "N": 0.5j * np.pi * k * k * a * dJ * dH,
    }


def _errors(a, k, N, modes):
    g = nodes(W.circle(a), N)
    ops = layer_operators(g, k)
    out = {}
    for key, A in ops.items():
        e = 0.0
        for m in modes:
            lam = A[0, :] @ np.exp(1j * m * g.t)
            ref = _closed(a, k, m)[key]
            e = max(e, abs(lam - ref) / max(1.0, abs(ref)))
        out[key] = e
    return out


@pytest.mark.parametrize("a,k", [(1.0, 3.0), (0.8, 3.0 - 0.4j), (1.0, 0.5 + 0.2j)])
def test_circle_eigenvalue_rates(a, k):
    modes = [0, 1, 2, 5]
    e64 = _errors(a, k, 64, modes)
    e256 = _errors(a, k, 256, modes)
    for key in ("S", "D", "Ds"):
        assert e256[key] < 1e-5, (key, e256[key])
        assert e64[key] / e256[key] > 14.0, (key, e64[key], e256[key])      # at least O(h^2)
    assert e256["N"] < 0.1 * (1 + abs(k) ** 2)
    assert 3.0 < e64["N"] / e256["N"] < 6.0                                   # O(h), as stated


def test_circulant_and_symmetry():
    g = nodes(W.circle(1.0), 48)
    ops = layer_operators(g, 2.0 + 0.1j)
    for A in ops.values():
        assert np.allclose(A[1:, 1:], A[:-1, :-1], atol=1e-13)             # circulant
    assert np.allclose(ops["S"], ops["S"].T, atol=1e-14)                   # S symmetric (equal weights)
    assert np.allclose(ops["D"], ops["Ds"], atol=1e-14)                    # D = D* on a circle


def test_trapezoid_identities_behind_the_corrections():
    # Exact finite sums that fix the one-point weights (log: prod 2 sin(pi j/N) = N;
    # hypersingular: sum 1/sin^2(pi j/N) = (N^2-1)/3).
    for N in (8, 33, 256):
        j = np.arange(1, N)
        assert abs(np.sum(np.log(2 * np.sin(np.pi * j / N))) - np.log(N)) < 1e-11
        assert abs(np.sum(1 / np.sin(np.pi * j / N) ** 2) - (N * N - 1) / 3) < 1e-8 * N * N


def test_calderon_weak():
    # D S = S D* holds exactly for the continuous operators (§2.2 Calderon relations);
    # on a non-circular curve the discrete defect shrinks with N.
    defects = []
    for N in (64, 128, 256):
        g = nodes(W.ellipse(1.0, 0.6), N)
        o = layer_operators(g, 2.0)
        defects.append(np.abs(o["D"] @ o["S"] - o["S"] @ o["Ds"]).max())
    assert defects[2] < defects[1] < defects[0]
    assert defects[0] / defects[2] > 3.5

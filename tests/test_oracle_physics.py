"""Physics pins for the oracle: the Bessel-series (Mie) solution of §5.1 with the O(1/N) rate the
paper states, the circle eigen-relation of §5.3, energy (optical theorem) and reciprocity of the
far field, and agreement between the mixed (Eq. dis_mixedBM) and ordinary (Eq. dis_BM) systems."""
import numpy as np
import pytest
from scipy import special as sp

import workloads as W
import oracle as O
from oracle.dense import schur_solve


def _relerr(X, N, u, q):
    num = np.linalg.norm(np.concatenate([X[:N] - u, X[N:2 * N] - q]))
    return num / np.linalg.norm(np.concatenate([u, q]))


def _solve_circle(N, k0, k1, literal=False):
    g = O.nodes(W.circle(1.0), N)
    P = O.default_params(k0, k1)
    blocks = O.mixed_blocks(g, P)
    Xm = schur_solve(blocks, O.rhs_plane_wave(g, P, [0.0], W.MIXED))[:, 0]
    Ao = O.ordinary_matrix(g, P, literal_ordinary=literal)
    Xo = O.dense_solve(Ao, O.rhs_plane_wave(g, P, [0.0], W.ORDINARY))[:, 0]
    u, q = O.mie_boundary(1.0, P.k0, P.k1, P.eps0, P.eps1, g.t)
    return g, P, Xm, Xo, u, q


def test_mie_first_order_convergence_both_formulations():
    # Eq. norm of §5.1 on [u; q]; the paper reports O(N^-1) for both formulations.
    errs_m, errs_o = [], []
    for N in (64, 128, 256):
        g, P, Xm, Xo, u, q = _solve_circle(N, 2.0, 3.0)
        errs_m.append(_relerr(Xm, N, u, q))
        errs_o.append(_relerr(Xo, N, u, q))
    for e in (errs_m, errs_o):
        assert e[-1] < 1e-2
        assert 1.8 < e[0] / e[1] < 2.2 and 1.8 < e[1] / e[2] < 2.2


@pytest.mark.parametrize("omega, eps1", [(1.0, 2.0), (2.0, 5.0), (10.0, 10.0)])
def test_mie_convergence_at_the_lu_experiment_parameters(omega, eps1):
    # §5.1, Table tb:lu_parameters: unit circle, eps0 = 1, the three (omega, eps1) pairs, the
    # first two sizes N = 100 * 2^i (i = 1, 2) and the plane wave exp(i k0 x1).  Fig. convLU_error
    # shows both formulations approaching the Bessel-series solution at O(N^-1): the Eq. norm error
    # halves from N = 200 to 400 for every pair, and on the circle the two systems give the same
    # [u; q] to rounding.
    errs_m, errs_o = [], []
    for N in (200, 400):
        g, P, Xm, Xo, u, q = _solve_circle(N, omega, omega * np.sqrt(eps1))
        assert abs(P.eps1 - eps1) < 1e-12 and P.eps0 == 1.0
        errs_m.append(_relerr(Xm, N, u, q))
        errs_o.append(_relerr(Xo, N, u, q))
        assert np.linalg.norm(Xm[:2 * N] - Xo) / np.linalg.norm(Xo) < 1e-11
    for e in (errs_m, errs_o):
        assert e[1] < 0.05
        assert 1.9 < e[0] / e[1] < 2.1, e


def test_literal_ordinary_reading_does_not_converge():
    g, P, Xm, Xl, u, q = _solve_circle(256, 2.0, 3.0, literal=True)
    assert _relerr(Xl, 256, u, q) > 0.3


def test_mixed_equals_ordinary_on_circle():
    g, P, Xm, Xo, u, q = _solve_circle(256, 2.0, 3.0)
    assert np.linalg.norm(Xm[:512] - Xo) / np.linalg.norm(Xo) < 1e-12


def test_mixed_vs_ordinary_on_ellipse_is_discretisation_error():
    diffs = []
    for N in (64, 128, 256):
        g = O.nodes(W.ellipse(1.0, 0.6), N)
        P = O.default_params(2.0, 3.0)
        Xm = schur_solve(O.mixed_blocks(g, P), O.rhs_plane_wave(g, P, [0.0], W.MIXED))[:, 0]
        Xo = O.dense_solve(O.ordinary_matrix(g, P), O.rhs_plane_wave(g, P, [0.0], W.ORDINARY))[:, 0]
        diffs.append(np.linalg.norm(Xm[:2 * N] - Xo) / np.linalg.norm(Xo))
    assert diffs[0] > 1e-9                           # genuinely different discretisations
    assert diffs[0] / diffs[1] > 4 and diffs[1] / diffs[2] > 4


def test_mie_series_determinant_is_paper_eigen_relation():
    # First circle eigen-relation of §5.3:
    #   -eps0 k1 H_n(k0 a) J_n'(k1 a) + eps1 k0 H_n'(k0 a) J_n(k1 a)
    # equals eps0*eps1 times the determinant of the 2x2 transmission system.
    a, k0, k1, e0, e1 = 0.5, 1.3 - 0.2j, 2.6 - 0.4j, 1.0, 4.0
    for n in range(0, 6):
        Hn, dHn = sp.hankel1(n, k0 * a), sp.h1vp(n, k0 * a)
        Jn, dJn = sp.jv(n, k1 * a), sp.jvp(n, k1 * a)
        paper = -e0 * k1 * Hn * dJn + e1 * k0 * dHn * Jn
        det = Hn * (-(k1 / e1) * dJn) - (-Jn) * ((k0 / e0) * dHn)
        assert abs(paper - e0 * e1 * det) < 1e-12 * abs(paper)


def test_mie_coefficients_lossless_energy():
    # |2 c_m + 1| = 1 for a lossless scatterer (c_m = a_m (-i)^m): per-mode optical theorem.
    m, am, bm = O.mie_coefficients(1.0, 2.0, 3.0, 1.0, 2.25)
    c = am * (-1j) ** m
    assert np.abs(np.abs(2 * c + 1) - 1).max() < 1e-13


def test_far_field_quadrature_of_mie_data_matches_closed_form():
    # Trapezoid rule on smooth periodic data is spectrally accurate: pins the far-field formula.
    a, k0, k1, e0, e1 = 1.0, 2.0, 3.0, 1.0, 2.25
    g = O.nodes(W.circle(a), 128)
    u, q = O.mie_boundary(a, k0, k1, e0, e1, g.t)
    th = np.linspace(0, 2 * np.pi, 17)
    F = O.far_field(g, k0, e0, u, q, th)
    Fr = O.mie_far_field(a, k0, k1, e0, e1, th)
    assert np.abs(F - Fr).max() < 1e-12 * np.abs(Fr).max()


def _ff_ellipse(N, angle, obs):
    g = O.nodes(W.ellipse(1.0, 0.6), N)
    P = O.default_params(2.0, 3.0)
    X = schur_solve(O.mixed_blocks(g, P), O.rhs_plane_wave(g, P, [angle], W.MIXED))[:, 0]
    return O.far_field(g, P.k0, P.eps0, X[:N], X[N:2 * N], obs), P


def test_optical_theorem_and_reciprocity_tighten_with_N():
    th = 2 * np.pi * np.arange(256) / 256
    defects, recips = [], []
    for N in (64, 128, 256):
        F, P = _ff_ellipse(N, 0.3, th)
        F0, _ = _ff_ellipse(N, 0.3, np.array([0.3]))
        lhs = np.sum(np.abs(F) ** 2) * (2 * np.pi / 256)
        rhs = -np.sqrt(8 * np.pi / 2.0) * np.real(np.exp(0.25j * np.pi) * F0[0])
        defects.append(abs(lhs - rhs) / abs(rhs))
        # reciprocity u_inf(xhat; dhat) = u_inf(-dhat; -xhat)
        Fa, _ = _ff_ellipse(N, 0.3, np.array([1.9]))
        Fb, _ = _ff_ellipse(N, 1.9 + np.pi, np.array([0.3 + np.pi]))
        recips.append(abs(Fa[0] - Fb[0]) / abs(Fa[0]))
    # both defects are discretisation errors: first order in h, like the solution error
    assert defects[-1] < 3e-3 and recips[-1] < 1e-3
    for e in (defects, recips):
        assert 1.8 < e[0] / e[1] < 2.2 and 1.8 < e[1] / e[2] < 2.2


def test_near_singular_at_paper_eigenvalue():
    # §5.3 / Table tb:ssm_eigenvalues: circle a = 0.5, eps1 = 4, omega* zero of H_2 -> the mixed
    # operator is singular at omega*; the discrete smallest singular value dips there.
    ws = 0.4294849652 - 1.2813737977j
    g = O.nodes(W.circle(0.5), 96)

    def smin(w):
        P = O.default_params(w, 2 * w, eps0=1.0, eps1=4.0)
        return np.linalg.svd(O.mixed_matrix(O.mixed_blocks(g, P)), compute_uv=False)[-1]

    s0 = smin(ws)
    s1 = smin(ws + 0.05)
    s2 = smin(ws - 0.05j)
    assert s0 < 0.15 * min(s1, s2), (s0, s1, s2)


def test_row_builders_match_the_assembled_systems():
    # The entry-by-entry row builders (used for sampled checks at full size) reproduce rows of the
    # dense systems, which the Mie-series pins above tie to the physics; ellipse, complex k,
    # eps1 != 1, rows from every block row including the diagonal entries.
    curve, N = W.ellipse(1.0, 0.6), 48
    g = O.nodes(curve, N)
    P = O.default_params(3.0 - 0.2j, 4.5 - 0.3j)
    A = O.mixed_matrix(O.mixed_blocks(g, P))
    rows = [0, 7, N - 1, N, N + 13, 2 * N - 1, 2 * N, 2 * N + 21, 3 * N - 1]
    assert np.abs(O.mixed_rows(g, P, rows) - A[rows]).max() <= 1e-14 * np.abs(A).max()
    Ao = O.ordinary_matrix(g, P)
    rows = [0, 5, N - 1, N, N + 30, 2 * N - 1]
    assert np.abs(O.ordinary_rows(g, P, rows) - Ao[rows]).max() <= 1e-14 * np.abs(Ao).max()

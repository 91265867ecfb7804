"""Pins for the oracle's high-order zeta-corrected rule (oracle/zeta.py; §4 quadrature, §5.3 "order
31" rule).

* The weights against things other than themselves: the log weights against a 40-digit mpmath
  evaluation of zeta'(-2k) and the same moment equations; the rule on two periodic model
  integrals with exact values,
      int_0^2pi ln(4 sin^2((t-s)/2)) e^{ims} ds = -2pi/|m| e^{imt}          (log singularity)
      f.p. int_0^2pi e^{ims} / (4 sin^2((t-s)/2)) ds = -pi |m| e^{imt}      (x^-2 singularity),
  converging at O(h^(2p+3)) and O(h^(2p+3)) (with the (p+1)-point second-derivative stencil).
  A wrong zeta value, sign or stencil weight leaves a lower order.
* The operators: circle eigenvalues against the closed forms (Graf's addition theorem), the ellipse
  against a fine-grid reference, and the Mie-series solution, all at order 2p+3 for S, D, D*, N.
* The paper's own check (Table tb:ssm_eigenvalues): with the order-31 rule (p = 14) the contour
  eigensolver finds the double eigenvalue at the zero of H_2^(1) to the digits the table prints,
  for both formulations, at N = 64.
"""
import os

import numpy as np
import pytest
from scipy import special as sp

import workloads as W
import oracle as O
from oracle import zeta, ssm
from oracle.dense import schur_solve

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hankel_zeros.txt")


def _order(e):
    return [np.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]


def _model_log(N, p, m=3):
    h = 2 * np.pi / N
    x = h * np.arange(1, N)
    val = h * np.sum(np.log(4 * np.sin(x / 2) ** 2) * np.exp(1j * m * x))
    tau = zeta.log_weights(p)
    # ln(4 sin^2(x/2)) = 2 ln|x| + smooth, smooth part 0 at x = 0
    val += 2.0 * h * (np.log(h / (2 * np.pi)) - 2 * sum(tau))
    for q, t in enumerate(tau, start=1):
        val += 2.0 * h * t * 2 * np.cos(m * q * h)
    return abs(val + 2 * np.pi / m)


def _model_hyper(N, p, m=3):
    h = 2 * np.pi / N
    x = h * np.arange(1, N)
    val = h * np.sum(np.exp(1j * m * x) / (4 * np.sin(x / 2) ** 2)) - np.pi ** 2 / (3 * h)
    c = zeta.second_derivative_weights(p + 1)
    s = c[0] * 1.0
    for q in range(1, p + 2):
        for xq in (q * h, -q * h):
            s += c[q] * xq * xq * np.exp(1j * m * xq) / (4 * np.sin(xq / 2) ** 2)
    return abs(val + s / (2 * h) + np.pi * m)


def test_log_weights_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for p in (1, 4, 9):
        tau = zeta.log_weights(p)
        A = mp.matrix([[mp.mpf(m) ** (2 * k) for m in range(1, p + 1)] for k in range(1, p + 1)])
        b = mp.matrix([mp.zeta(-2 * k, derivative=1) for k in range(1, p + 1)])
        ref = mp.lu_solve(A, b)
        for m in range(p):
            assert abs(tau[m] - float(ref[m])) <= 1e-14 * abs(float(ref[m]))


def test_second_derivative_stencil_exact_on_polynomials():
    for q in (1, 3, 6):
        c = zeta.second_derivative_weights(q)
        for deg in range(0, 2 * q + 2):
            est = c[0] * (1.0 if deg == 0 else 0.0) + sum(c[m] * (m ** deg + (-m) ** deg) for m in range(1, q + 1))
            assert abs(est - (2.0 if deg == 2 else 0.0)) < 1e-9


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_model_integrals_converge_at_order_2p_plus_3(p):
    Ns = (32, 64, 128)
    el = [_model_log(N, p) for N in Ns]
    assert min(_order(el)) > 2 * p + 3 - 0.3, el
    if p > 0:
        eh = [_model_hyper(N, p) for N in Ns]
        assert min(_order(eh)) > 2 * p + 3 - 0.3, eh


def _closed(a, k, m):
    z = k * a
    J, dJ = sp.jv(m, z), sp.jvp(m, z)
    H, dH = sp.hankel1(m, z), sp.h1vp(m, z)
    return {"S": 0.5j * np.pi * a * J * H, "D": 0.25j * np.pi * k * a * (dJ * H + J * dH),
            "Ds": 0.25j * np.pi * k * a * (dJ * H + J * dH), "N": 0.5j * np.pi * k * k * a * dJ * dH}


@pytest.mark.parametrize("p", [1, 2])
def test_circle_eigenvalues_at_order_2p_plus_3(p):
    a, k = 1.0, 3.0 - 0.4j
    errs = {key: [] for key in ("S", "D", "Ds", "N")}
    for N in (32, 64, 128):
        g = O.nodes(W.circle(a), N)
        ops = O.layer_operators(g, k, p)
        for key, A in ops.items():
            e = 0.0
            for m in (0, 1, 2, 5):
                ref = _closed(a, k, m)[key]
                e = max(e, abs(A[0, :] @ np.exp(1j * m * g.t) - ref) / max(1.0, abs(ref)))
            errs[key].append(e)
    for key, e in errs.items():
        assert _order(e)[-1] > 2 * p + 3 - 0.5, (key, e)


def test_corrections_touch_only_the_stencil_band():
    g = O.nodes(W.ellipse(1.0, 0.6), 40)
    base = O.layer_operators(g, 2.0, 0)
    hi = O.layer_operators(g, 2.0, 2)
    i, j = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    dist = np.minimum(np.abs(i - j), 40 - np.abs(i - j))
    for key in base:
        changed = np.abs(hi[key] - base[key]) > 0
        assert not changed[dist > 3].any(), key
    assert (np.abs(hi["S"] - base["S"])[dist == 2] > 0).all()       # log stencil: |m| <= p
    assert not (np.abs(hi["S"] - base["S"])[dist == 3] > 0).any()
    assert (np.abs(hi["N"] - base["N"])[dist == 3] > 0).all()       # N: |m| <= p + 1


def test_ellipse_self_convergence():
    curve, k, p = W.ellipse(1.0, 0.6), 4.0 + 0.3j, 2

    def apply(N, q):
        g = O.nodes(curve, N)
        phi = np.exp(2j * g.t) * (1 + 0.3 * np.cos(3 * g.t))
        return {key: A @ phi for key, A in O.layer_operators(g, k, q).items()}

    ref = apply(512, 6)
    errs = {key: [] for key in ref}
    for N in (64, 128):
        r = apply(N, p)
        for key in r:
            errs[key].append(np.abs(r[key] - ref[key][::512 // N]).max() / np.abs(ref[key]).max())
    for key, e in errs.items():
        assert _order(e)[0] > 2 * p + 3 - 0.5, (key, e)


@pytest.mark.parametrize("p", [1, 2])
def test_mie_solution_at_order_2p_plus_3(p):
    errs = []
    for N in (32, 64, 128):
        g = O.nodes(W.circle(1.0), N)
        P = O.default_params(2.0, 3.0)
        X = schur_solve(O.mixed_blocks(g, P, p), O.rhs_plane_wave(g, P, [0.0], W.MIXED))[:, 0]
        u, q = O.mie_boundary(1.0, P.k0, P.k1, P.eps0, P.eps1, g.t)
        errs.append(np.linalg.norm(np.concatenate([X[:N] - u, X[N:2 * N] - q])) / np.linalg.norm(np.concatenate([u, q])))
    assert _order(errs)[-1] > 2 * p + 3 - 0.5, errs


def _table():
    out = {}
    for line in open(GOLD):
        f = line.split()
        if f and not f[0].startswith("#") and f[0] == "2":
            out[f[1]] = complex(float(f[2]), float(f[3]))
    return out


def test_order_31_rule_reproduces_the_paper_table():
    # Table tb:ssm_eigenvalues: Doring's zero to 10 digits, and the paper's own order-31 runs to
    # ~1e-12 of each other; p = 14 is order 2p + 3 = 31
    tab = _table()
    target = tab["reference_doring"]
    N = 64
    for form, key, nsys in ((W.MIXED, "mixed_run1", 3 * N), (W.ORDINARY, "ordinary_run1", 2 * N)):
        V = W.gaussian_full(nsys, 4, 3)
        inside, _, _ = ssm.ssm(W.circle(0.5), N, 2.0, form, target, 0.05, 32, 4, V, 1e-10, zeta_p=14)
        assert inside.size == 2
        assert np.abs(inside - target).max() < 6e-11          # the table's 10 printed digits
        assert np.abs(inside - tab[key]).max() < 2e-11        # the paper's computed value


@pytest.mark.parametrize("p,order", [(0, 1), (3, 9)])
def test_calderon_identities_on_the_ellipse(p, order):
    # Calderon relations (§2.2): S N = D^2 - I/4 and N S = D*^2 - I/4 for the same wavenumber.
    # Applied to a smooth density the discrete defect vanishes at the rule's order (O(h) with the
    # one-point rule, whose N is first order; O(h^(2p+3)) with the corrections), which ties N to S
    # and D on a non-circular curve.
    errs = []
    for N in (64, 128, 256):
        g = O.nodes(W.ellipse(1.0, 0.6), N)
        o = O.layer_operators(g, 2.0 + 0.1j, p)
        phi = np.exp(2j * g.t) * (1 + 0.3 * np.cos(3 * g.t))
        d1 = np.abs(o["S"] @ (o["N"] @ phi) - (o["D"] @ (o["D"] @ phi) - 0.25 * phi)).max()
        d2 = np.abs(o["N"] @ (o["S"] @ phi) - (o["Ds"] @ (o["Ds"] @ phi) - 0.25 * phi)).max()
        errs.append(max(d1, d2) / np.abs(phi).max())
    assert min(_order(errs)) > order - 0.3, errs

"""GPU parity at the full workload sizes, on outputs the oracle computes one at a time.

Star r = 1 + 0.3 cos 5t, N = 4096 (the benchmark system: 12288 unknowns, 65 RHS) and kite, N = 16384
(49152 unknowns, 8 RHS), each in the launch configuration the benchmark uses.  The full matrices are
far too large for the oracle, so each test checks what it can evaluate entry by entry:

* assembled blocks at 3000 sampled (i, j) pairs (diagonal ones included) against the oracle's
  operator entries, 1e-12 of the largest sampled entry (as the small-N assembly tests);
* the plane-wave right-hand side against the oracle, 1e-13;
* the solution through the residual of sampled rows, r_i = b_i - A_i x with the rows built by the
  oracle: max |r_i| / (a ||x||_inf + ||b||_inf) per column, with a = the largest sampled row sum
  (a lower bound of ||A||_inf, so the check is at least as strict as the backward error).  Bound:
  2e-9 after refinement (the library certifies 1e-9 with the exact ||A||_inf), 1e-12 for FP64;
* the far field at sampled angles against the oracle's sum, 1e-12.
"""
import numpy as np
import pytest

import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


def _rhs(g, P, w, form):
    Bp = O.rhs_plane_wave(g, P, [0.0], form)
    G = W.place_rhs(W.gaussian_g(w.N, w.n_gauss, w.seed), w.N, form)
    return np.asfortranarray(np.concatenate([Bp, G], 1))


def _check_blocks(bm, h, torch, g, P, N):
    rng = np.random.default_rng(11)
    I = rng.integers(0, N, 3000)
    J = rng.integers(0, N, 3000)
    J[:200] = I[:200]
    e = (I == J).astype(float)
    o0 = O.layer_entries(g, P.k0, I, J)
    o1 = O.layer_entries(g, P.k1, I, J)
    ref = [-o1["S"], -(o1["Ds"] + 0.5 * e) / P.eps1, o0["D"] - 0.5 * e + P.beta * o0["N"],
           -P.eps0 * (o0["S"] + P.beta * (o0["Ds"] + 0.5 * e))]
    M = torch.empty((N, N), dtype=torch.complex128, device="cuda").t()
    ti, tj = torch.as_tensor(I, device="cuda"), torch.as_tensor(J, device="cuda")
    for which in range(4):
        bm.bm_copy_block(h, which, M)
        got = M[ti, tj].cpu().numpy()
        err = np.abs(got - ref[which]).max() / np.abs(ref[which]).max()
        assert err < 1e-12, (which, err)
    del M


def _sampled_eta(rows_fn, g, P, rows, X, B):
    A = rows_fn(g, P, rows)
    R = B[rows] - A @ X
    a = np.abs(A).sum(1).max()
    den = a * np.abs(X).max(0) + np.abs(B).max(0)
    return float((np.abs(R).max(0) / den).max())


def _rows(N, nblk, per):
    rng = np.random.default_rng(5)
    return np.concatenate([b * N + rng.choice(N, per, replace=False) for b in range(nblk)] + [[0, nblk * N - 1]])


def _solve_case(bm, w, form, prec, check_blocks):
    torch = pytest.importorskip("torch")
    N = w.N
    g = O.nodes(w.curve, N)
    P = O.default_params(w.k_out, w.k_in)
    h = bm.bm_create(0)
    try:
        bm.bm_assemble(h, w.curve.kind, w.curve.params4(), N, w.k_out, w.k_in, form, bm.make_opts(prec))
        if check_blocks:
            _check_blocks(bm, h, torch, g, P, N)
        assert bm.bm_factor(h) == 0
        B = _rhs(g, P, w, form)
        Bl = np.zeros((B.shape[0], 1), dtype=np.complex128, order="F")
        bm.bm_rhs_plane_wave(h, [0.0], Bl)
        assert np.abs(Bl[:, 0] - B[:, 0]).max() <= 1e-13 * np.abs(B[:, 0]).max()
        X = np.zeros_like(B, order="F")
        info = bm.bm_solve(h, B, X)
        assert np.isfinite(X).all()
        if prec != bm.BM_FP64:
            assert info.backward_error <= 1e-9
        nblk = 3 if form == bm.BM_MIXED else 2
        eta = _sampled_eta(O.mixed_rows if form == bm.BM_MIXED else O.ordinary_rows, g, P, _rows(N, nblk, 6), X, B)
        assert eta <= (1e-12 if prec == bm.BM_FP64 else 2e-9), eta
        th = np.linspace(0.0, 2.0 * np.pi, 16, endpoint=False)
        U = np.zeros((th.size, X.shape[1]), dtype=np.complex128, order="F")
        bm.bm_far_field(h, X, th, U)
        Ur = O.far_field(g, P.k0, P.eps0, X[:N], X[N:2 * N], th)
        assert np.abs(U - Ur).max() <= 1e-12 * np.abs(Ur).max()
        return X
    finally:
        bm.bm_destroy(h)


@pytest.mark.parametrize("form", [0, 1])
def test_star_n4096_3xtf32_refined(bmlib, form):
    _solve_case(bmlib, W.STAR_N4096, form, bmlib.BM_CF32_3XTF32_IR, check_blocks=(form == 0))


def test_star_n4096_fp64_and_tf32_agree(bmlib):
    w = W.STAR_N4096
    X64 = _solve_case(bmlib, w, 0, bmlib.BM_FP64, check_blocks=False)
    X32 = _solve_case(bmlib, w, 0, bmlib.BM_CF32_TF32_IR, check_blocks=False)
    # both are backward stable at ~1e-14 / 1e-9: the difference is conditioning times that
    assert np.linalg.norm(X64 - X32) / np.linalg.norm(X64) < 1e-6


@pytest.mark.parametrize("form", [0, 1])
def test_kite_n16384_3xtf32_refined(bmlib, form):
    _solve_case(bmlib, W.KITE_N16384, form, bmlib.BM_CF32_3XTF32_IR, check_blocks=(form == 0))


def test_kite_n16384_fp64(bmlib):
    _solve_case(bmlib, W.KITE_N16384, 0, bmlib.BM_FP64, check_blocks=False)

"""GPU parity: factor + solve of both systems against the oracle.

FP64 path: relative 2-norm error of the whole solution vector (3N or 2N) <= 1e-10 against the
oracle's solve of the same right-hand sides (Theorem thm:LU / Corollary lem:for_ssm_RHS path for
the mixed system, full dense LU for the ordinary one).
Mixed-precision paths: backward error <= 1e-9 as reported by the library AND as recomputed by
the oracle with its own FP64 operator; solution within 1e-9 * cond-scale of the oracle's.
Sizes span several LU panels and a ragged tail (N = 200: U33 200 x 200 with 128-wide panels;
ordinary N = 500: 1000 x 1000, which spreads each panel over a 2-CTA cluster)."""
import numpy as np
import pytest

import workloads as W
import oracle as O
from oracle.dense import schur_solve


def _setup(bmlib, handle, curve, N, k0, k1, form, prec):
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, form, bmlib.make_opts(prec))
    info = bmlib.bm_factor(handle)
    assert info == 0
    g = O.nodes(curve, N)
    P = O.default_params(k0, k1)
    return g, P


def _rhs(g, P, N, form, n_gauss, full=False, seed=0):
    Bp = O.rhs_plane_wave(g, P, [0.0, 0.7], form)
    nsys = Bp.shape[0]
    if full:
        G = W.gaussian_full(nsys, n_gauss, seed)
    else:
        G = W.place_rhs(W.gaussian_g(N, n_gauss, seed), N, form)
    return np.asfortranarray(np.concatenate([Bp, G], 1))


def _relerr(X, Xr):
    return np.linalg.norm(X - Xr) / np.linalg.norm(Xr)


@pytest.mark.gpu
@pytest.mark.parametrize("curve,N,k0,k1", [(W.star(1.0, 0.3, 5), 200, 6.0, 9.0),
                                            (W.ellipse(1.0, 0.6), 150, 5.0 - 0.2j, 7.5 - 0.3j)])
def test_fp64_mixed_matches_oracle(bmlib, handle, curve, N, k0, k1):
    g, P = _setup(bmlib, handle, curve, N, k0, k1, bmlib.BM_MIXED, bmlib.BM_FP64)
    B = _rhs(g, P, N, W.MIXED, 5, full=True)      # b1, b2 != 0 exercises the Corollary
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    Xr = schur_solve(O.mixed_blocks(g, P), B)
    assert _relerr(X, Xr) < 1e-10
    assert info.backward_error < 1e-13


@pytest.mark.gpu
def test_fp64_mixed_matches_full_dense_definition(bmlib, handle):
    curve, N = W.kite(), 70
    g, P = _setup(bmlib, handle, curve, N, 4.0, 6.0, bmlib.BM_MIXED, bmlib.BM_FP64)
    B = _rhs(g, P, N, W.MIXED, 2)
    X = np.zeros_like(B, order="F")
    bmlib.bm_solve(handle, B, X)
    Xr = O.dense_solve(O.mixed_matrix(O.mixed_blocks(g, P)), B)   # unblocked LU of the full 3N matrix
    assert _relerr(X, Xr) < 1e-10


@pytest.mark.gpu
@pytest.mark.parametrize("N", [150, 500])
def test_fp64_ordinary_matches_oracle(bmlib, handle, N):
    curve = W.star(1.0, 0.25, 4)
    g, P = _setup(bmlib, handle, curve, N, 5.0, 7.5, bmlib.BM_ORDINARY, bmlib.BM_FP64)
    B = _rhs(g, P, N, W.ORDINARY, 3)
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    Xr = O.dense_solve(O.ordinary_matrix(g, P), B)
    assert _relerr(X, Xr) < 1e-10
    assert info.backward_error < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("resid", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("form", [0, 1])
def test_mixed_precision_refinement(bmlib, handle, prec, form, resid):
    # first residual from tensor-core digit products (0), FP64 (1) or double-float (3), later ones
    # r -= A d in FP32; 2: every residual in FP64
    curve, N, k0, k1 = W.star(1.0, 0.3, 5), 200, 6.0, 9.0
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, form,
                      bmlib.make_opts(prec, residual=resid))
    assert bmlib.bm_factor(handle) == 0
    g, P = O.nodes(curve, N), O.default_params(k0, k1)
    B = _rhs(g, P, N, form, 6, full=(form == 0))
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    assert info.backward_error <= 1e-9
    assert info.iterations >= 1
    if form == W.MIXED:
        blocks = O.mixed_blocks(g, P)
        eta = O.backward_error_mixed(blocks, X, B)
        Xr = schur_solve(blocks, B)
    else:
        A = O.ordinary_matrix(g, P)
        eta = O.backward_error_dense(A, X, B)
        Xr = O.dense_solve(A, B)
    assert eta <= 1.5e-9
    assert _relerr(X, Xr) < 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("clmax,N,kernel", [(1, 600, ""), (1, 1100, ""), (2, 1100, ""), (2, 500, ""),
                                            (16, 1100, "rows")])
def test_panel_variants_match_oracle(bmlib, prec, clmax, N, kernel):
    # Capping the panel cluster puts 2 (N=600, cap 1; N=1100, cap 2) or 4 (N=1100, cap 1) rows on
    # each thread of the register-row panel kernel, which selects its narrower sub-panel variants;
    # FP32 panels of at most 256 rows per CTA run on the lane-per-column kernel (N=500, cap 2: 16
    # rows per warp).  kernel="rows" keeps every FP32 panel on the register-row kernel.
    h = bmlib.bm_create(0)
    try:
        curve, k0, k1 = W.ellipse(1.0, 0.6), 6.0 - 0.1j, 9.0 - 0.15j
        opts = bmlib.make_opts(prec, panel_cluster_max=clmax, panel_kernel=1 if kernel == "rows" else 0)
        bmlib.bm_assemble(h, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_MIXED, opts)
        assert bmlib.bm_factor(h) == 0
        g, P = O.nodes(curve, N), O.default_params(k0, k1)
        B = _rhs(g, P, N, W.MIXED, 3, full=True, seed=5)
        X = np.zeros_like(B, order="F")
        info = bmlib.bm_solve(h, B, X)
        blocks = O.mixed_blocks(g, P)
        if prec == 0:
            assert _relerr(X, schur_solve(blocks, B)) < 1e-10
        else:
            assert info.backward_error <= 1e-9
            assert O.backward_error_mixed(blocks, X, B) <= 1.5e-9
    finally:
        bmlib.bm_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("resid", [0, 3])
@pytest.mark.parametrize("form", [0, 1])
def test_first_residual_reaches_tight_tolerance(bmlib, handle, form, resid):
    # Refinement can only certify what its residual resolves: reaching 2e-12 through the
    # tensor-core digit residual (0) or the double-float one (3), and FP32 updates, pins that
    # residual far below the 1e-9 target.
    curve, N, k0, k1 = W.kite(), 300, 9.0 - 0.2j, 13.5 - 0.3j
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, form,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, refine_tol=2e-12, residual=resid))
    assert bmlib.bm_factor(handle) == 0
    g, P = O.nodes(curve, N), O.default_params(k0, k1)
    B = _rhs(g, P, N, form, 4, full=(form == 0), seed=3)
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    assert info.backward_error <= 2e-12
    eta = (O.backward_error_mixed(O.mixed_blocks(g, P), X, B) if form == 0
           else O.backward_error_dense(O.ordinary_matrix(g, P), X, B))
    assert eta <= 5e-12


@pytest.mark.gpu
def test_mixed_and_ordinary_agree_on_circle(bmlib, handle):
    # On a circle the two discretisations agree to rounding (all matrices circulant, D = D*).
    N = 256
    out = []
    for form in (bmlib.BM_MIXED, bmlib.BM_ORDINARY):
        bmlib.bm_assemble(handle, W.CIRCLE, (1.0, 0, 0), N, 2.0, 3.0, form, bmlib.make_opts())
        assert bmlib.bm_factor(handle) == 0
        nsys = 3 * N if form == bmlib.BM_MIXED else 2 * N
        B = np.zeros((nsys, 1), dtype=np.complex128, order="F")
        bmlib.bm_rhs_plane_wave(handle, [0.0], B)
        X = np.zeros_like(B, order="F")
        bmlib.bm_solve(handle, B, X)
        out.append(X[:2 * N, 0])
    assert np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[1]) < 1e-12
    # and both sit at the O(1/N) distance from the Bessel-series solution (section 5.1)
    P = O.default_params(2.0, 3.0)
    u, q = O.mie_boundary(1.0, P.k0, P.k1, P.eps0, P.eps1, O.nodes(W.circle(1.0), N).t)
    ref = np.concatenate([u, q])
    e = np.linalg.norm(out[0] - ref) / np.linalg.norm(ref)
    assert 5e-3 < e < 8e-3


@pytest.mark.gpu
def test_far_field_matches_oracle(bmlib, handle):
    curve, N = W.ellipse(1.0, 0.6), 120
    g, P = _setup(bmlib, handle, curve, N, 3.0 - 0.1j, 4.5 - 0.15j, bmlib.BM_MIXED, bmlib.BM_FP64)
    B = _rhs(g, P, N, W.MIXED, 1)
    X = np.zeros_like(B, order="F")
    bmlib.bm_solve(handle, B, X)
    th = np.linspace(0, 2 * np.pi, 33)
    U = np.zeros((th.size, X.shape[1]), dtype=np.complex128, order="F")
    bmlib.bm_far_field(handle, X, th, U)
    Ur = O.far_field(g, P.k0, P.eps0, X[:N], X[N:2 * N], th)
    assert np.abs(U - Ur).max() / np.abs(Ur).max() < 1e-12


@pytest.mark.gpu
def test_far_field_many_columns_and_ragged_angles(bmlib, handle):
    # more columns than one CTA takes (two column tiles of the node contraction), an angle count
    # that is not a multiple of the 8-angle tile, and enough nodes for 8-CTA clusters of node slices
    curve, N = W.ellipse(1.0, 0.6), 600
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 3.0 - 0.1j, 4.5 - 0.15j, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_FP64))
    g, P = O.nodes(curve, N), O.default_params(3.0 - 0.1j, 4.5 - 0.15j)
    X = np.asfortranarray(W.gaussian_full(3 * N, 130, 5))
    th = np.linspace(0.1, 2 * np.pi + 0.1, 70, endpoint=False)
    U = np.zeros((th.size, X.shape[1]), dtype=np.complex128, order="F")
    bmlib.bm_far_field(handle, X, th, U)
    Ur = O.far_field(g, P.k0, P.eps0, X[:N], X[N:2 * N], th)
    assert np.abs(U - Ur).max() / np.abs(Ur).max() < 1e-12


@pytest.mark.gpu
def test_device_arrays_and_repeat_calls(bmlib, handle):
    torch = pytest.importorskip("torch")
    curve, N = W.circle(1.0), 128
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 2.0, 3.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR))
    assert bmlib.bm_factor(handle) == 0
    assert bmlib.bm_factor(handle) == 0            # cached graph replay gives the same factors
    Bd = torch.zeros((2, 3 * N), dtype=torch.complex128, device="cuda").t()
    bmlib.bm_rhs_plane_wave(handle, [0.0, 1.0], Bd)
    Xd = torch.zeros((2, 3 * N), dtype=torch.complex128, device="cuda").t()
    i1 = bmlib.bm_solve(handle, Bd, Xd)
    X1 = Xd.cpu().numpy().copy()
    i2 = bmlib.bm_solve(handle, Bd, Xd)
    assert i1.backward_error <= 1e-9 and i2.backward_error <= 1e-9
    assert np.array_equal(X1, Xd.cpu().numpy())    # deterministic
    Bh = np.asfortranarray(Bd.cpu().numpy())
    Xh = np.zeros_like(Bh, order="F")
    bmlib.bm_solve(handle, Bh, Xh)
    assert np.array_equal(X1, Xh)


@pytest.mark.gpu
def test_profile_reports_every_kernel_and_the_same_solution(bmlib, handle):
    # bm_profile runs the factorisation and solve with every launch timed: the solution is the one a
    # normal call gives, and the groups cover the method's kernels with positive times
    curve, N = W.star(1.0, 0.3, 5), 600
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 6.0, 9.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR))
    assert bmlib.bm_factor(handle) == 0
    B = np.asfortranarray(W.gaussian_full(3 * N, 3, 2))
    X1 = np.zeros_like(B, order="F")
    bmlib.bm_solve(handle, B, X1)
    X2 = np.zeros_like(B, order="F")
    prof = bmlib.bm_profile(handle, B, X2)
    assert np.array_equal(X1, X2)
    names = {k for k, _, _ in prof}
    for k in ("cgemm_tc_kernel (Schur complement)", "panel_lc_kernel", "cgemm_tc_kernel (trailing update)",
              "trsv_flow_kernel", "resid_tc_kernel (+ split-K reduction)", "eta_kernel"):
        assert k in names, k
    assert all(l >= 1 and ms > 0 for _, l, ms in prof)
    assert [ms for _, _, ms in prof] == sorted([ms for _, _, ms in prof], reverse=True)


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 33, 70])
def test_tensor_core_residual_ragged_shapes(bmlib, handle, form, nrhs):
    # N = 150: K = 150 and 300 end inside a 64-wide K block and a 256-wide exact chunk; 1, 33 and 70
    # right-hand sides end inside a 32-wide column tile (a 16-wide last product).  The refined
    # solution is certified to 2e-12 through the digit residual, and the oracle's FP64 backward
    # error agrees.
    curve, N, k0, k1 = W.ellipse(1.0, 0.6), 150, 5.0 - 0.1j, 7.5 - 0.15j
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, form,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, refine_tol=2e-12, residual=0))
    assert bmlib.bm_factor(handle) == 0
    g, P = O.nodes(curve, N), O.default_params(k0, k1)
    nsys = 3 * N if form == 0 else 2 * N
    B = np.asfortranarray(W.gaussian_full(nsys, nrhs, 7))
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    assert info.backward_error <= 2e-12
    eta = (O.backward_error_mixed(O.mixed_blocks(g, P), X, B) if form == 0
           else O.backward_error_dense(O.ordinary_matrix(g, P), X, B))
    assert eta <= 5e-12


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1])
def test_nine_digit_residual_refines_to_fp64_accuracy(bmlib, handle, form):
    # every residual afresh from nine-digit tensor-core products: TF32 factors refined to 1e-14
    # (beyond what FP32-updated residuals can certify), confirmed by the oracle's FP64 residual
    curve, N, k0, k1 = W.kite(), 300, 9.0 - 0.2j, 13.5 - 0.3j
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, form,
                      bmlib.make_opts(bmlib.BM_CF32_TF32_IR, refine_tol=1e-14, residual=bmlib.BM_RESID_TC_ALL))
    assert bmlib.bm_factor(handle) == 0
    g, P = O.nodes(curve, N), O.default_params(k0, k1)
    B = _rhs(g, P, N, form, 5, full=(form == 0), seed=4)
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    assert info.backward_error <= 1e-14
    eta = (O.backward_error_mixed(O.mixed_blocks(g, P), X, B) if form == 0
           else O.backward_error_dense(O.ordinary_matrix(g, P), X, B))
    assert eta <= 3e-14

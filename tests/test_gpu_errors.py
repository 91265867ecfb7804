"""GPU-side error behaviour of the C ABI: call order, invalid arguments, non-finite input and
HBM-budget admission.  None of these faults the GPU: every failure is detected on the host or
by a device reduction and returned as a status."""
import time

import numpy as np
import pytest

import workloads as W


@pytest.mark.gpu
def test_call_order(bmlib, handle):
    B = np.zeros((24, 1), dtype=np.complex128, order="F")
    X = np.zeros_like(B, order="F")
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_factor(handle)
    assert e.value.status == bmlib.BM_ESTATE
    bmlib.bm_assemble(handle, W.CIRCLE, (1.0, 0, 0), 8, 2.0, 3.0, bmlib.BM_MIXED, bmlib.make_opts())
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_solve(handle, B, X)
    assert e.value.status == bmlib.BM_ESTATE


@pytest.mark.gpu
def test_invalid_arguments(bmlib, handle):
    for args in [(W.CIRCLE, (1.0, 0, 0), 4, 2.0, 3.0),        # N too small
                 (W.CIRCLE, (-1.0, 0, 0), 64, 2.0, 3.0),      # negative radius
                 (W.CIRCLE, (1.0, 0, 0), 64, -2.0, 3.0),      # Re k <= 0
                 (W.STAR, (1.0, 1.5, 5), 64, 2.0, 3.0)]:      # self-intersecting star
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_assemble(handle, *args, bmlib.BM_MIXED, bmlib.make_opts())
        assert e.value.status == bmlib.BM_EINVAL
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_assemble(handle, W.CIRCLE, (1.0, 0, 0), 64, float("nan"), 3.0, bmlib.BM_MIXED, bmlib.make_opts())
    assert e.value.status == bmlib.BM_ENONFINITE


@pytest.mark.gpu
def test_nonfinite_rhs(bmlib, handle):
    N = 32
    bmlib.bm_assemble(handle, W.CIRCLE, (1.0, 0, 0), N, 2.0, 3.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_TF32_IR))
    bmlib.bm_factor(handle)
    B = np.ones((3 * N, 1), dtype=np.complex128, order="F")
    B[5, 0] = np.nan
    X = np.zeros_like(B, order="F")
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_solve(handle, B, X)
    assert e.value.status == bmlib.BM_ENONFINITE


@pytest.mark.gpu
def test_budget_admission(bmlib):
    h = bmlib.bm_create(0, None, 64 << 20)   # 64 MB budget
    try:
        held0, budget = bmlib.bm_memory(h)
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_assemble(h, W.CIRCLE, (1.0, 0, 0), 2048, 2.0, 3.0, bmlib.BM_MIXED, bmlib.make_opts())
        assert e.value.status == bmlib.BM_ENOMEM
        assert bmlib.bm_memory(h)[0] == held0     # nothing was allocated
        bmlib.bm_assemble(h, W.CIRCLE, (1.0, 0, 0), 256, 2.0, 3.0, bmlib.BM_MIXED, bmlib.make_opts())
        assert bmlib.bm_memory(h)[0] <= budget
    finally:
        bmlib.bm_destroy(h)


@pytest.mark.gpu
def test_tight_tolerance_needs_fp64_residuals(bmlib, handle):
    # updated residuals are only trusted to ~1e-12: a tighter target with them is refused
    curve = W.circle(1.0)
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_assemble(handle, curve.kind, curve.params4(), 64, 2.0, 3.0, bmlib.BM_MIXED,
                          bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, refine_tol=1e-14, residual=0))
    assert e.value.status == bmlib.BM_EINVAL
    for resid in (bmlib.BM_RESID_FP64_ALL, bmlib.BM_RESID_TC_ALL):
        bmlib.bm_assemble(handle, curve.kind, curve.params4(), 64, 2.0, 3.0, bmlib.BM_MIXED,
                          bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, refine_tol=1e-14, residual=resid))


@pytest.mark.gpu
def test_refinement_cap_reports_not_converged(bmlib, handle):
    # one TF32 correction cannot reach 1e-12: BM_ENOTCONV, with the last iterate in X
    curve, N = W.kite(), 200
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 6.0, 9.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_TF32_IR, refine_tol=1e-12, refine_maxit=1))
    assert bmlib.bm_factor(handle) == 0
    B = np.zeros((3 * N, 1), dtype=np.complex128, order="F")
    bmlib.bm_rhs_plane_wave(handle, [0.0], B)
    X = np.zeros_like(B, order="F")
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_solve(handle, B, X)
    assert e.value.status == bmlib.BM_ENOTCONV
    info = bmlib.bm_solve(handle, B, X, raise_on_notconv=False)
    assert info.iterations == 1 and 1e-12 < info.backward_error < 1e-3
    assert np.isfinite(X).all() and np.abs(X).max() > 0
    # the handle goes on: a looser target on the same factors converges
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 6.0, 9.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_TF32_IR))
    assert bmlib.bm_factor(handle) == 0
    assert bmlib.bm_solve(handle, B, X).backward_error <= 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1])
def test_device_wait_timeout_is_reported_and_the_device_stays_usable(bmlib, form):
    # The test hook makes every tensor-core product wait on a barrier nothing completes; the wait
    # gives up after ~1 ms, the product skips its output, and bm_factor reports BM_ETIMEOUT.  No
    # kernel is left running: the same handle and a fresh one then factor and solve correctly.
    curve, N = W.ellipse(1.0, 0.6), 300
    nsys = 3 * N if form == 0 else 2 * N
    h = bmlib.bm_create(0)
    try:
        bmlib.bm_assemble(h, curve.kind, curve.params4(), N, 5.0, 7.5, form,
                          bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, test_wait_timeout=True))
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_factor(h)
        assert e.value.status == bmlib.BM_ETIMEOUT
        B = np.zeros((nsys, 1), dtype=np.complex128, order="F")
        X = np.zeros_like(B, order="F")
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_solve(h, B, X)                  # not factored
        assert e.value.status == bmlib.BM_ESTATE
        for hh in (h, None):
            g = hh if hh is not None else bmlib.bm_create(0)
            try:
                bmlib.bm_assemble(g, curve.kind, curve.params4(), N, 5.0, 7.5, form,
                                  bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR))
                assert bmlib.bm_factor(g) == 0
                bmlib.bm_rhs_plane_wave(g, [0.0], B)
                assert bmlib.bm_solve(g, B, X).backward_error <= 1e-9
            finally:
                if hh is None:
                    bmlib.bm_destroy(g)
    finally:
        bmlib.bm_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1])
def test_triangular_solve_wait_timeout_is_reported(bmlib, form):
    # Hook 2: one wait of the persistent triangular solve is on a flag nothing sets; it gives up
    # after ~1 s, the rest of that launch stops waiting, and bm_solve reports BM_ETIMEOUT at its
    # next read-back instead of iterating.  The handle then factors and solves correctly again.
    curve, N = W.ellipse(1.0, 0.6), 300
    nsys = 3 * N if form == 0 else 2 * N
    h = bmlib.bm_create(0)
    try:
        bmlib.bm_assemble(h, curve.kind, curve.params4(), N, 5.0, 7.5, form,
                          bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, test_wait_timeout=2))
        assert bmlib.bm_factor(h) == 0
        B = np.zeros((nsys, 2), dtype=np.complex128, order="F")
        bmlib.bm_rhs_plane_wave(h, [0.0, 1.0], B)
        X = np.zeros_like(B, order="F")
        t0 = time.time()
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_solve(h, B, X)
        assert e.value.status == bmlib.BM_ETIMEOUT
        assert time.time() - t0 < 20.0
        bmlib.bm_assemble(h, curve.kind, curve.params4(), N, 5.0, 7.5, form,
                          bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR))
        assert bmlib.bm_factor(h) == 0
        assert bmlib.bm_solve(h, B, X).backward_error <= 1e-9
    finally:
        bmlib.bm_destroy(h)


@pytest.mark.gpu
def test_nonfinite_far_field_angles(bmlib, handle):
    torch = pytest.importorskip("torch")
    N = 64
    bmlib.bm_assemble(handle, W.CIRCLE, (1.0, 0, 0), N, 2.0, 3.0, bmlib.BM_MIXED, bmlib.make_opts())
    assert bmlib.bm_factor(handle) == 0
    X = torch.zeros((1, 3 * N), dtype=torch.complex128, device="cuda").t()
    U = torch.zeros((1, 3), dtype=torch.complex128, device="cuda").t()
    for fn in (bmlib.bm_far_field, bmlib.bm_far_field_static):
        with pytest.raises(bmlib.BMError) as e:
            fn(handle, X, [0.0, float("inf"), 1.0], U)
        assert e.value.status == bmlib.BM_ENONFINITE

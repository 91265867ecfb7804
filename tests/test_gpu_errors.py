"""GPU-side error behaviour of the C ABI: call order, invalid arguments, non-finite input and
HBM-budget admission.  None of these faults the GPU: every failure is detected on the host or
by a device reduction and returned as a status."""
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
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), 64, 2.0, 3.0, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, refine_tol=1e-14, residual=2))

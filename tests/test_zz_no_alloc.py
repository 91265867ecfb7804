"""bm_far_field_static (no device allocation) against bm_far_field on the same solution.

bm_far_field_static stages the observation angles in a fixed device array built into the
library instead of a buffer allocated per call; the far-field kernel is the same.  The file name
puts it last in collection, so it also runs after every other GPU test of the session.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N, NRHS = 120, 3
REL_TOL = 1e-13  # same kernel on the same data: equal up to nothing but the angles' source


def _solution(bm, h, torch):
    curve = W.ellipse(1.0, 0.6)
    bm.bm_assemble(h, curve.kind, curve.params4(), N, 3.0 - 0.1j, 4.5 - 0.15j, bm.BM_MIXED, bm.make_opts())
    assert bm.bm_factor(h) == 0
    B = torch.zeros((NRHS, 3 * N), dtype=torch.complex128, device="cuda").t()
    bm.bm_rhs_plane_wave(h, np.linspace(0.0, 1.0, NRHS), B)
    X = torch.zeros((NRHS, 3 * N), dtype=torch.complex128, device="cuda").t()
    bm.bm_solve(h, B, X)
    return X


def _far(bm, h, torch, X, th, static):
    U = torch.full((NRHS, th.size), complex("nan"), dtype=torch.complex128, device="cuda").t()
    (bm.bm_far_field_static if static else bm.bm_far_field)(h, X, th, U)
    return U.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_static_far_field_matches_far_field_on_consecutive_calls(bmlib, handle):
    torch = pytest.importorskip("torch")
    X = _solution(bmlib, handle, torch)
    th1 = np.linspace(0.0, 2.0 * np.pi, 257)
    th2 = np.linspace(0.3, 1.3, 40)  # fewer angles: nothing of the first call may leak in
    ref1 = _far(bmlib, handle, torch, X, th1, static=False)
    ref2 = _far(bmlib, handle, torch, X, th2, static=False)
    held0 = bmlib.bm_memory(handle)[0]
    got1 = _far(bmlib, handle, torch, X, th1, static=True)
    got2 = _far(bmlib, handle, torch, X, th2, static=True)
    assert np.isfinite(got1).all() and np.isfinite(got2).all()
    assert _rel(got1, ref1) <= REL_TOL
    assert _rel(got2, ref2) <= REL_TOL
    # the handle allocated nothing for these calls
    assert bmlib.bm_memory(handle)[0] == held0


def test_static_far_field_size_limit(bmlib, handle):
    torch = pytest.importorskip("torch")
    X = _solution(bmlib, handle, torch)
    M = bmlib.BM_FAR_FIELD_STATIC_MAX_ANGLES
    th = np.linspace(0.0, 2.0 * np.pi, M, endpoint=False)
    assert _rel(_far(bmlib, handle, torch, X, th, static=True),
                _far(bmlib, handle, torch, X, th, static=False)) <= REL_TOL
    th_big = np.linspace(0.0, 2.0 * np.pi, M + 1)
    U = torch.zeros((NRHS, M + 1), dtype=torch.complex128, device="cuda").t()
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_far_field_static(handle, X, th_big, U)
    assert e.value.status == bmlib.BM_EINVAL
    assert str(M) in str(e.value)

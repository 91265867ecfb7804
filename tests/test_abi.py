"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/bm.h declares,
its host-built Hankel anchor and Taylor tables match scipy and its high-order zeta weights match the
oracle's, and its argument checks run before any device work (no GPU needed for any of this)."""
import os
import re

import numpy as np
import pytest
from scipy import special as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(bmlib):
    import ctypes
    L = ctypes.CDLL(bmlib.LIB_PATH)
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_every_exported_entry_point_is_declared(bmlib):
    # the other direction: no bm_* symbol leaves the library without a declaration in bm.h
    import shutil
    import subprocess
    if shutil.which("nm") is None:
        pytest.skip("nm is not installed")
    out = subprocess.run(["nm", "-D", "--defined-only", bmlib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("bm_")})
    assert exported
    assert sorted(set(exported) - set(_declared())) == []


def test_strerror_names_every_status(bmlib):
    for s in range(9):
        assert bmlib.bm_strerror(s).startswith("BM_")


def test_anchor_table_matches_scipy(bmlib):
    T, re0, im0, step = bmlib.bm_hankel_anchor_table()
    ny, nx, _ = T.shape
    iy, ix = np.mgrid[0:ny, 0:nx]
    z = re0 + ix * step + 1j * (im0 + iy * step)
    used = (np.abs(z) >= 2.75) & (np.abs(z) <= 80.25)      # anchors the device Taylor zone can pick
    H0, H1 = sp.hankel1(0, z[used]), sp.hankel1(1, z[used])
    e = np.maximum(np.abs(T[..., 0][used] - H0) / np.abs(H0), np.abs(T[..., 1][used] - H1) / np.abs(H1))
    assert used.sum() > 150000
    assert e.max() < 1e-14


def test_taylor_table_reproduces_scipy(bmlib):
    # the coefficients the device Taylor zone evaluates, summed by Horner's scheme with the
    # derivative (H1 = -H0') at the nearest anchor, over the zone 3 <= |z| < 80, arg -70..60 deg
    T, re0, im0, step = bmlib.bm_hankel_anchor_table()
    A = bmlib.bm_hankel_taylor_table()
    assert A.shape[:2] == T.shape[:2] and A.shape[2] >= 12
    np.testing.assert_array_equal(A[..., 0], T[..., 0])       # a_0 = H0(z0)
    np.testing.assert_array_equal(A[..., 1], -T[..., 1])      # a_1 = -H1(z0)
    rng = np.random.default_rng(7)
    r = np.concatenate([3.0 + 77.0 * rng.random(6000), [3.0, 20.0, 79.999999]])
    th = np.radians(rng.uniform(-70.0, 60.0, r.size))
    z = r * np.exp(1j * th)
    ix = np.rint((z.real - re0) / step).astype(int)
    iy = np.rint((z.imag - im0) / step).astype(int)
    d = z - (re0 + ix * step + 1j * (im0 + iy * step))
    assert np.abs(d).max() <= step / np.sqrt(2) + 1e-12
    c = A[iy, ix]
    p = c[:, -1].copy()
    q = np.zeros_like(p)
    for k in range(c.shape[1] - 2, -1, -1):
        q = q * d + p
        p = p * d + c[:, k]
    H0, H1 = sp.hankel1(0, z), sp.hankel1(1, z)
    assert np.max(np.abs(p - H0) / np.abs(H0)) < 1e-14
    assert np.max(np.abs(-q - H1) / np.abs(H1)) < 1e-14


def test_create_without_gpu_reports_cuda_error(bmlib):
    import torch
    if torch.cuda.is_available():
        return
    import ctypes
    h = ctypes.c_void_p()
    st = bmlib.lib().bm_create(ctypes.byref(h), 0, None, 0)
    assert st == bmlib.BM_ECUDA


def test_contour_and_server_argument_checks_need_no_gpu(bmlib):
    # bm_ssm and bm_server_create check their arguments before touching the device
    import ctypes
    import numpy as np
    cv = bmlib.bm_curve()
    cv.kind = bmlib.BM_CURVE_CIRCLE
    cv.p[0] = 1.0
    so = bmlib.bm_ssm_opts()
    so.center = bmlib.bm_c64(5.0, 0.0)
    so.radius = 0.5
    so.npoints = 32
    so.nmoments = 4
    so.k_ratio = bmlib.bm_c64(1.5, 0.0)
    N, L = 64, 4
    V = np.zeros((3 * N, L), dtype=np.complex128, order="F")
    om = np.zeros(L * 4, dtype=np.complex128)
    info = bmlib.bm_ssm_info()

    def call(so_, L_=L, cap=L * 4, ldv=3 * N):
        return bmlib.lib().bm_ssm(0, ctypes.byref(cv), N, bmlib.BM_MIXED, None, ctypes.byref(so_),
                                  ctypes.c_void_p(V.ctypes.data), ldv, L_, ctypes.c_void_p(om.ctypes.data), cap,
                                  None, ctypes.byref(info))

    for field, bad in (("radius", 0.0), ("npoints", 2), ("nmoments", 0), ("nmoments", 17), ("workers", 65),
                       ("batch", 65), ("panel_cluster", 17), ("batch", -1),
                       ("rank_tol", 1.5)):
        s2 = bmlib.bm_ssm_opts.from_buffer_copy(so)
        setattr(s2, field, bad)
        assert call(s2) == bmlib.BM_EINVAL, field
    assert call(so, cap=L * 4 - 1) == bmlib.BM_EINVAL          # output too small for L M eigenvalues
    assert call(so, ldv=3 * N - 1) == bmlib.BM_EINVAL          # leading dimension below the system size
    assert call(so, L_=65) == bmlib.BM_EINVAL                  # L M above 256
    o = bmlib.bm_server_opts()
    o.slots = 0
    srv = ctypes.c_void_p()
    assert bmlib.lib().bm_server_create(ctypes.byref(srv), 0, ctypes.byref(o)) == bmlib.BM_EINVAL
    o.slots = 33
    assert bmlib.lib().bm_server_create(ctypes.byref(srv), 0, ctypes.byref(o)) == bmlib.BM_EINVAL


def test_zeta_order_and_block_solve_argument_checks_need_no_gpu(bmlib):
    # the quadrature order is checked before any device work (bm_ssm validates its bm_opts), and
    # bm_solve_block rejects a missing handle
    import ctypes
    import numpy as np
    cv = bmlib.bm_curve()
    cv.kind = bmlib.BM_CURVE_CIRCLE
    cv.p[0] = 0.5
    so = bmlib.bm_ssm_opts()
    so.center = bmlib.bm_c64(0.43, -1.28)
    so.radius = 0.05
    so.npoints = 32
    so.nmoments = 4
    so.k_ratio = bmlib.bm_c64(2.0, 0.0)
    N, L = 64, 4
    V = np.zeros((3 * N, L), dtype=np.complex128, order="F")
    om = np.zeros(L * 4, dtype=np.complex128)
    info = bmlib.bm_ssm_info()
    for p in (-1, 21, 31):                        # 31: N = 64 < 2 p + 3
        o = bmlib.make_opts(zeta_p=p)
        st = bmlib.lib().bm_ssm(0, ctypes.byref(cv), N, bmlib.BM_MIXED, ctypes.byref(o), ctypes.byref(so),
                                ctypes.c_void_p(V.ctypes.data), 3 * N, L, ctypes.c_void_p(om.ctypes.data), L * 4,
                                None, ctypes.byref(info))
        assert st == bmlib.BM_EINVAL, p
    X = np.zeros((3 * N, 1), dtype=np.complex128, order="F")
    st = bmlib.lib().bm_solve_block(None, 1, ctypes.c_void_p(X.ctypes.data), 3 * N, 0, None, 1, 0, None, 1,
                                    ctypes.c_void_p(X.ctypes.data), 3 * N, 0, None)
    assert st == bmlib.BM_EINVAL


def test_library_zeta_weights_match_the_oracle(bmlib):
    # the library builds the high-order correction weights on the host with a construction of its
    # own (Euler-Maclaurin zeta(2k+1), Bjorck-Pereyra Vandermonde solve, closed-form stencil);
    # the oracle's come from scipy's zeta and exact rational elimination
    import numpy as np
    from oracle import zeta
    for p in (1, 2, 5, 14, 20):
        tau, c2 = bmlib.bm_zeta_weights(p)
        ref_tau = np.array(zeta.log_weights(p))
        assert np.abs(tau[1:] - ref_tau).max() <= 1e-14 * np.abs(ref_tau).max()
        assert abs(tau[0] + 2 * ref_tau.sum()) <= 1e-14
        ref_c2 = np.array(zeta.second_derivative_weights(p + 1))
        assert np.abs(c2 - ref_c2).max() <= 1e-13 * np.abs(ref_c2).max()
    with pytest.raises(bmlib.BMError):
        bmlib.bm_zeta_weights(21)


def test_binding_rejects_outputs_too_small_for_the_write(bmlib):
    # The library sees leading dimensions only; the binding checks that U has a column per solution
    # and a row per angle (and X the system's rows) before any call, so no device write can run past
    # an array.  No handle or GPU is needed: the checks fire first.
    import torch
    X = torch.zeros((3, 30), dtype=torch.complex128).t()          # 30 x 3 (host tensors)
    th = np.linspace(0.0, 1.0, 7)
    for U in (torch.zeros((2, 7), dtype=torch.complex128).t(),     # too few columns
              torch.zeros((3, 6), dtype=torch.complex128).t()):    # too few rows
        with pytest.raises(ValueError):
            bmlib.bm_far_field(None, X, th, U)
        with pytest.raises(ValueError):
            bmlib.bm_far_field_static(None, X, th, U)
    B = np.zeros((30, 2), dtype=np.complex128, order="F")
    with pytest.raises(ValueError):
        bmlib.bm_rhs_plane_wave(None, [0.0, 1.0, 2.0], B)          # a column per angle
    with pytest.raises(ValueError):
        bmlib.bm_solve(None, B, np.zeros((30, 3), dtype=np.complex128, order="F"))
    # bm_copy_block writes the whole block: dst must have its rows and its columns
    key = bmlib._hkey(None)
    bmlib._blk[key] = 30
    try:
        for shape in ((30, 29), (29, 30), (30, 1)):
            with pytest.raises(ValueError):
                bmlib.bm_copy_block(None, 0, np.zeros(shape, dtype=np.complex128, order="F"))
            with pytest.raises(ValueError):
                bmlib.bm_copy_block(None, 0, torch.zeros(shape[::-1], dtype=torch.complex128).t())
    finally:
        bmlib._blk.pop(key, None)


def test_binding_holds_serving_arrays_until_collected(bmlib, monkeypatch):
    # A queued request's worker reads B and writes X on another thread until the request is
    # collected, so the binding keeps both arrays alive until bm_server_wait (or bm_server_destroy)
    # returns, whatever the caller does with its own references.  A stand-in library records the
    # calls; no GPU is needed.
    import ctypes
    import gc
    import weakref

    class FakeLib:
        def bm_server_submit(self, s, req, ticket):
            ctypes.cast(ticket, ctypes.POINTER(ctypes.c_ulonglong))[0] = 7
            return bmlib.BM_OK

        def bm_server_wait(self, s, ticket, res):
            return bmlib.BM_OK

        def bm_server_destroy(self, s):
            return bmlib.BM_OK

    monkeypatch.setattr(bmlib, "lib", lambda: FakeLib())
    s = ctypes.c_void_p(12345)
    B = np.ones((24, 2), dtype=np.complex128, order="F")
    X = np.zeros((24, 2), dtype=np.complex128, order="F")
    refs = [weakref.ref(B), weakref.ref(X)]
    t = bmlib.bm_server_submit(s, 0, (1.0, 0, 0, 0), 8, 2.0, 3.0, bmlib.BM_MIXED, B, X)
    assert t == 7
    del B, X
    gc.collect()
    assert all(r() is not None for r in refs)          # still held while in flight
    bmlib.bm_server_wait(s, t)
    gc.collect()
    assert all(r() is None for r in refs)              # released once collected
    B = np.ones((24, 1), dtype=np.complex128, order="F")
    r2 = weakref.ref(B)
    bmlib.bm_server_submit(s, 0, (1.0, 0, 0, 0), 8, 2.0, 3.0, bmlib.BM_MIXED, B,
                           np.zeros((24, 1), dtype=np.complex128, order="F"))
    del B
    bmlib.bm_server_destroy(s)                          # every request has finished by then
    gc.collect()
    assert r2() is None and not bmlib._in_flight

"""GPU parity: device Hankel functions and Nystrom assembly against the oracle (FP64 both sides).

Tolerances: Hankel 2e-14 relative per point (the three device zones are each accurate to a
few 1e-15; scipy's own error is ~1e-15); assembled entries 1e-12 of the block's largest entry
(the entries are sums of a few Hankel-based terms; the oracle uses scipy's AMOS Hankel)."""
import numpy as np
import pytest

import workloads as W
import oracle as O


def _zpoints():
    # every zone and both sides of each boundary (series | Taylor at 3, Taylor | asymptotic at 80)
    r = np.concatenate([np.geomspace(1e-5, 2.99, 40), [2.9999999, 3.0, 3.0000001], np.linspace(3.01, 19.99, 120),
                        [19.9999999, 20.0, 20.0000001], np.linspace(20.01, 79.99, 120),
                        [79.9999999, 80.0, 80.0000001], np.geomspace(80.01, 600.0, 30)])
    ang = np.deg2rad([-70.0, -30.0, -10.0, -2.0, 0.0, 3.0, 20.0, 45.0, 60.0])
    z = (r[:, None] * np.exp(1j * ang[None, :])).ravel()
    return z[np.abs(z.imag) <= 60.0]


@pytest.mark.gpu
def test_device_hankel_all_zones(bmlib, handle):
    z = _zpoints()
    h0, h1 = bmlib.bm_hankel01(handle, z)
    r0, r1 = O.hankel01(z)
    e0 = np.abs(h0 - r0) / np.abs(r0)
    e1 = np.abs(h1 - r1) / np.abs(r1)
    worst = np.argmax(np.maximum(e0, e1))
    assert max(e0.max(), e1.max()) < 2e-14, (z[worst], e0[worst], e1[worst])


@pytest.mark.gpu
def test_device_fp32_conversions_match_ieee(bmlib, handle):
    # the integer FP64 -> FP32 rounding (row norms) against numpy's IEEE conversion: random
    # magnitudes over the FP32 range and beyond, ties and near-ties of the 29 dropped bits, binade
    # and range edges, values whose result is subnormal or overflows (the fallback path)
    rng = np.random.default_rng(13)
    x = [rng.standard_normal(100000) * 10.0 ** rng.uniform(-45, 40, 100000)]
    base = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)).view(np.uint64) & ~np.uint64((1 << 29) - 1)
    for off in (0, 1, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, (1 << 29) - 1):
        x.append((base | np.uint64(off)).view(np.float64))
    x.append(np.array([0.0, -0.0, 1.0, -1.0, 3.4e38, 1.1754943508222875e-38, 1e-39, 1e-45, 1e-300,
                       2.0 ** -126, 2.0 ** -126 * (1 - 2 ** -30), 2.0 ** 127, 1 + 2 ** -24, 1 + 3 * 2 ** -25]))
    x = np.concatenate(x)
    rn = bmlib.bm_f32_convert(handle, x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(rn.view(np.uint32), ref.view(np.uint32))


CASES = [
    (W.circle(1.0), 64, 2.0, 3.0),
    (W.ellipse(1.0, 0.6), 100, 5.0 - 0.3j, 7.5 - 0.45j),
    (W.star(1.0, 0.3, 5), 130, 20.0, 30.0),
    (W.kite(0.65, 1.5), 97, 11.0, 16.5),
    (W.circle(0.5), 40, 0.4294849652 - 1.2813737977j, 2 * (0.4294849652 - 1.2813737977j)),
]


def _oracle_blocks(curve, N, k0, k1, eps1=None):
    g = O.nodes(curve, N)
    P = O.default_params(k0, k1, eps1=eps1)
    return g, P


@pytest.mark.gpu
@pytest.mark.parametrize("curve,N,k0,k1", CASES)
def test_mixed_blocks_match_oracle(bmlib, handle, curve, N, k0, k1):
    eps1 = 4.0 if N == 40 else None
    opts = bmlib.make_opts(bmlib.BM_FP64, eps1=eps1)
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_MIXED, opts)
    g, P = _oracle_blocks(curve, N, k0, k1, eps1)
    ref = O.mixed_blocks(g, P)
    for which in range(4):
        M = np.zeros((N, N), dtype=np.complex128, order="F")
        bmlib.bm_copy_block(handle, which, M)
        err = np.abs(M - ref[which]).max() / np.abs(ref[which]).max()
        assert err < 1e-12, (which, err)


@pytest.mark.gpu
@pytest.mark.parametrize("curve,N,k0,k1", CASES[:4])
def test_ordinary_matrix_matches_oracle(bmlib, handle, curve, N, k0, k1):
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_ORDINARY, bmlib.make_opts())
    g, P = _oracle_blocks(curve, N, k0, k1)
    ref = O.ordinary_matrix(g, P)
    A = np.zeros((2 * N, 2 * N), dtype=np.complex128, order="F")
    bmlib.bm_copy_block(handle, 0, A)
    assert np.abs(A - ref).max() / np.abs(ref).max() < 1e-12


@pytest.mark.gpu
def test_user_curve_equals_builtin(bmlib, handle):
    # a user-supplied node list of the star reproduces the built-in star exactly
    curve = W.star(1.0, 0.3, 5)
    N = 72
    g = O.nodes(curve, N)
    user = np.concatenate([g.x, g.dx, g.ddx], 1)  # x, y, x', y', x'', y''
    bmlib.bm_assemble(handle, bmlib.BM_CURVE_USER, (0, 0, 0, 0), N, 3.0, 4.5, bmlib.BM_MIXED, bmlib.make_opts(),
                      user=user)
    Mu = np.zeros((N, N), dtype=np.complex128, order="F")
    bmlib.bm_copy_block(handle, 2, Mu)
    ref = O.mixed_blocks(g, O.default_params(3.0, 4.5))[2]
    assert np.abs(Mu - ref).max() / np.abs(ref).max() < 1e-12


@pytest.mark.gpu
def test_plane_wave_rhs(bmlib, handle):
    curve, N = W.kite(), 90
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 7.0 - 0.2j, 10.5 - 0.3j, bmlib.BM_MIXED,
                      bmlib.make_opts())
    ang = [0.0, 1.1, -2.5]
    B = np.zeros((3 * N, 3), dtype=np.complex128, order="F")
    bmlib.bm_rhs_plane_wave(handle, ang, B)
    g = O.nodes(curve, N)
    ref = O.rhs_plane_wave(g, O.default_params(7.0 - 0.2j, 10.5 - 0.3j), ang, W.MIXED)
    assert np.abs(B - ref).max() / np.abs(ref).max() < 1e-13

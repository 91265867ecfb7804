"""GPU parity for the high-order zeta-corrected rule (bm_opts.zeta_p; §5.3's "order 31" rule, order
2p+3), against the oracle of oracle/zeta.py (its weights are pinned in tests/test_oracle_zeta.py).

* Assembled blocks: the mixed blocks M13, M23, M31, M32 and the ordinary 2N matrix equal the
  oracle's entry by entry (1e-12 of the block's largest entry) on the ellipse and the star with
  complex wavenumbers, for p = 1, 4 and 14.
* Solve: 3xTF32 + refinement with p = 4 gives the oracle's solution of the same system (backward
  error 1e-9, and the solution to 1e-7).
* The paper's check (Table tb:ssm_eigenvalues) on the device: the contour eigensolver with the
  order-31 rule (p = 14, N = 64, FP64) finds the double eigenvalue at the zero of H_2^(1) to the
  table's printed digits and to the paper's own order-31 values, for both formulations.
"""
import os

import numpy as np
import pytest

import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "hankel_zeros.txt")


@pytest.mark.parametrize("p", [1, 4, 14])
@pytest.mark.parametrize("curve,k0,k1", [(W.ellipse(1.0, 0.6), 3.0 - 0.2j, 4.5 - 0.3j),
                                         (W.star(1.0, 0.25, 4), 6.0, 9.0 - 0.1j)])
def test_blocks_match_oracle(bmlib, handle, curve, k0, k1, p):
    N = 64
    g = O.nodes(curve, N)
    P = O.default_params(k0, k1)
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_MIXED, bmlib.make_opts(zeta_p=p))
    ref = O.mixed_blocks(g, P, p)
    for which in range(4):
        M = np.zeros((N, N), dtype=np.complex128, order="F")
        bmlib.bm_copy_block(handle, which, M)
        err = np.abs(M - ref[which]).max() / np.abs(ref[which]).max()
        assert err < 1e-12, (which, err)
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_ORDINARY, bmlib.make_opts(zeta_p=p))
    A = np.zeros((2 * N, 2 * N), dtype=np.complex128, order="F")
    bmlib.bm_copy_block(handle, 0, A)
    refo = O.ordinary_matrix(g, P, zeta_p=p)
    assert np.abs(A - refo).max() / np.abs(refo).max() < 1e-12


def test_refined_solve_matches_oracle(bmlib, handle):
    curve, N, k0, k1, p = W.kite(), 96, 5.0 - 0.1j, 7.5 - 0.2j, 4
    g = O.nodes(curve, N)
    P = O.default_params(k0, k1)
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_MIXED,
                      bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR, zeta_p=p))
    assert bmlib.bm_factor(handle) == 0
    B = np.asfortranarray(W.gaussian_full(3 * N, 3, 5))
    X = np.zeros_like(B, order="F")
    info = bmlib.bm_solve(handle, B, X)
    assert info.backward_error <= 1e-9
    Xr = O.dense_solve(O.mixed_matrix(O.mixed_blocks(g, P, p)), B)
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) < 1e-7


def _table():
    out = {}
    for line in open(GOLD):
        f = line.split()
        if f and not f[0].startswith("#") and f[0] == "2":
            out[f[1]] = complex(float(f[2]), float(f[3]))
    return out


@pytest.mark.parametrize("form,key", [(0, "mixed_run1"), (1, "ordinary_run1")])
def test_order_31_contour_eigenvalues(bmlib, form, key):
    tab = _table()
    target = tab["reference_doring"]
    N = 64
    V = np.asfortranarray(W.gaussian_full(3 * N if form == 0 else 2 * N, 4, 3))
    curve = W.circle(0.5)
    om, sig, info = bmlib.bm_ssm(0, curve.kind, curve.params4(), N, form, bmlib.make_opts(bmlib.BM_FP64, zeta_p=14),
                                 target, 0.05, 32, 4, 2.0, V, rank_tol=1e-10)
    assert info.n_inside == 2
    got = om[:info.n_inside]
    assert np.abs(got - target).max() < 6e-11       # the table's 10 printed digits
    assert np.abs(got - tab[key]).max() < 2e-11     # the paper's order-31 value

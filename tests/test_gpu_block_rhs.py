"""GPU parity for bm_solve_block (Corollary lem:block_LU: the block-diagonal right-hand side
diag(B1, B2, B3) of the mixed system) against the oracle's literal form of the Corollary
(tests/test_oracle_dense.py pins that against LAPACK on the full 3N matrix).

* FP64: 1e-11 of the oracle's solution; 3xTF32 + refinement: backward error 1e-9 and the solution
  to 1e-7 (well-conditioned star).
* Host and device (torch) forms give identical results; an empty block drops its columns.
* The ordinary formulation has no block form: BM_ESTATE.
"""
import numpy as np
import pytest

import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


def _rand(n, m, seed):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.normal(size=(n, m)) + 1j * rng.normal(size=(n, m)))


@pytest.mark.parametrize("prec", [0, 2])
def test_block_rhs_matches_oracle(bmlib, handle, prec):
    torch = pytest.importorskip("torch")
    N, curve, k0, k1 = 64, W.star(1.0, 0.25, 4), 3.0 - 0.1j, 4.5
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, k0, k1, bmlib.BM_MIXED, bmlib.make_opts(prec))
    assert bmlib.bm_factor(handle) == 0
    B1, B2, B3 = _rand(N, 2, 1), _rand(N, 3, 2), _rand(N, 1, 3)
    X = np.zeros((3 * N, 6), dtype=np.complex128, order="F")
    info = bmlib.bm_solve_block(handle, B1, B2, B3, X)
    g = O.nodes(curve, N)
    blocks = O.mixed_blocks(g, O.default_params(k0, k1))
    Xr = O.block_rhs_solve(blocks, B1, B2, B3)
    rel = np.linalg.norm(X - Xr) / np.linalg.norm(Xr)
    assert rel < (1e-11 if prec == 0 else 1e-7), rel
    if prec != 0:
        assert info.backward_error <= 1e-9

    def dev(A):
        t = torch.zeros((A.shape[1], A.shape[0]), dtype=torch.complex128, device="cuda").t()
        t.copy_(torch.from_numpy(np.ascontiguousarray(A)))
        return t

    Xd = dev(np.zeros((3 * N, 6), dtype=np.complex128))
    bmlib.bm_solve_block(handle, dev(B1), dev(B2), dev(B3), Xd)
    assert np.array_equal(Xd.cpu().numpy(), X)
    X2 = np.zeros((3 * N, 4), dtype=np.complex128, order="F")
    bmlib.bm_solve_block(handle, None, B2, B3, X2)
    assert np.abs(X2 - Xr[:, 2:]).max() <= (1e-11 if prec == 0 else 1e-7) * np.abs(Xr).max()


def test_block_rhs_needs_the_mixed_system(bmlib, handle):
    N, curve = 32, W.circle(1.0)
    bmlib.bm_assemble(handle, curve.kind, curve.params4(), N, 2.0, 3.0, bmlib.BM_ORDINARY, bmlib.make_opts())
    assert bmlib.bm_factor(handle) == 0
    B = _rand(N, 1, 4)
    with pytest.raises(bmlib.BMError) as e:
        bmlib.bm_solve_block(handle, B, None, None, np.zeros((3 * N, 1), dtype=np.complex128, order="F"))
    assert e.value.status == bmlib.BM_ESTATE

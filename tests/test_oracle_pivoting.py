"""Where partial pivoting puts its pivots on the systems this library factors (no GPU).

The LU of Theorem thm:LU pivots by columns (the izamax rule: the first row of largest |Re| + |Im|
at or below the diagonal).  On the Schur complement U33 = -M31 M13 - M32 M23, and on the
ordinary 2N matrix of Eq. dis_BM, the oracle's unblocked LU takes the diagonal entry at every
step for the scatterers of the benchmark configurations.  The largest candidate below the
diagonal stays a fixed fraction of the pivot.  The ratio max_i |a_ik^(k)| / |a_kk^(k)| is at
most 0.48 for U33 and 0.89 for the ordinary matrix in the cases below, so no row is ever
interchanged.

This is a property of the operators, not a requirement of the library, whose panels keep the full
pivot search.  It is what lets a panel factor its columns on the assumption that every pivot is
on the diagonal, and check afterwards, exactly, that partial pivoting would have chosen the same
pivots (all candidates a_ik^(k) are formed on the way).  Where the check fails the panel is
factored again with the search."""
import numpy as np
import pytest

import workloads as W
import oracle as O
from oracle.dense import lu_factor, schur_complement


def _pivot_ratio(A):
    LU, piv = lu_factor(A)
    u = np.diag(LU)
    cand = np.tril(LU, -1) * u[None, :]          # a_ik^(k) = l_ik u_kk, i > k
    mag = np.abs(cand.real) + np.abs(cand.imag)
    ratio = mag.max(0)[:-1] / (np.abs(u.real) + np.abs(u.imag))[:-1]
    return int((piv != np.arange(A.shape[0])).sum()), float(ratio.max())


@pytest.mark.parametrize("curve, k0, k1", [
    (W.star(1.0, 0.3, 5), 20.0, 30.0),          # the benchmark scatterer
    (W.kite(), 100.0, 150.0),                    # the large single system's curve and wavenumbers
    (W.ellipse(1.0, 0.6), 5.5 - 0.3j, 8.25 - 0.45j),   # a contour-batch point (complex k)
    (W.circle(1.0), 2.0, 3.0),                   # the section 5.1 circle
])
def test_partial_pivoting_keeps_the_diagonal(curve, k0, k1):
    N = 256
    g = O.nodes(curve, N)
    P = O.default_params(k0, k1)
    swaps, ratio = _pivot_ratio(schur_complement(O.mixed_blocks(g, P)))
    assert swaps == 0 and ratio < 0.5, (swaps, ratio)
    swaps, ratio = _pivot_ratio(O.ordinary_matrix(g, P))
    assert swaps == 0 and ratio < 0.9, (swaps, ratio)


def test_pivot_ratio_sees_interchanges():
    # the measure itself: a matrix whose first column peaks below the diagonal does swap
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    A[0, 0] = 1e-3
    swaps, ratio = _pivot_ratio(A)
    assert swaps > 0 and ratio <= 1.0

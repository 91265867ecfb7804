"""Serving loop (bm_server): continuous batching of independent solves.

* Each result is the same in the mix as alone: ten requests of mixed shapes (star curves, N from
  48 to 128, complex wavenumbers, both formulations, 1..8 right-hand sides) submitted at once to a
  four-slot server give bit-identical solutions to the same requests run one after another on one
  handle - and they did overlap on the device.
* Every result is a correct solve: the oracle's backward error (FP64 path 1e-13, refined paths
  1.5e-9, as in the single-solve parity tests).
* Admission never lets the admitted bytes exceed the budget, and a request larger than the whole
  budget is refused at submission.
"""
import numpy as np
import pytest

import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


def _requests(n=10, seed=7):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        N = int(rng.choice([48, 64, 96, 128]))
        curve = W.star(1.0, float(rng.uniform(0.1, 0.3)), int(rng.integers(3, 9)))
        k = complex(rng.uniform(2.0, 12.0), rng.uniform(-0.5, 0.0))
        form = int(rng.integers(0, 2))
        nsys = 3 * N if form == W.MIXED else 2 * N
        B = np.asfortranarray(W.gaussian_full(nsys, int(rng.integers(1, 9)), 100 + i))
        reqs.append((curve, N, k, 1.5 * k, form, B))
    return reqs


@pytest.mark.parametrize("prec", [0, 2])
def test_results_alone_equal_results_in_the_mix(bmlib, prec):
    reqs = _requests()
    opts = bmlib.make_opts(prec)
    alone = []
    h = bmlib.bm_create(0)
    try:
        for curve, N, k0, k1, form, B in reqs:
            bmlib.bm_assemble(h, curve.kind, curve.params4(), N, k0, k1, form, opts)
            assert bmlib.bm_factor(h) == 0
            X = np.zeros_like(B, order="F")
            bmlib.bm_solve(h, B, X)
            alone.append(X)
    finally:
        bmlib.bm_destroy(h)
    s = bmlib.bm_server_create(0, slots=4, opts=opts)
    try:
        Xs = [np.zeros_like(r[5], order="F") for r in reqs]
        tickets = [bmlib.bm_server_submit(s, c.kind, c.params4(), N, k0, k1, form, B, X)
                   for (c, N, k0, k1, form, B), X in zip(reqs, Xs)]
        results = [bmlib.bm_server_wait(s, t) for t in tickets]
        st = bmlib.bm_server_stats_get(s)
    finally:
        bmlib.bm_server_destroy(s)
    assert st.completed == len(reqs) and st.max_in_flight > 1
    assert len({r.slot for r in results}) > 1
    for X, Xa in zip(Xs, alone):
        assert np.array_equal(X, Xa)
    for (curve, N, k0, k1, form, B), X in zip(reqs, Xs):
        g, P = O.nodes(curve, N), O.default_params(k0, k1)
        eta = (O.backward_error_mixed(O.mixed_blocks(g, P), X, B) if form == W.MIXED
               else O.backward_error_dense(O.ordinary_matrix(g, P), X, B))
        assert eta <= (1e-13 if prec == 0 else 1.5e-9)


def test_admission_respects_the_budget(bmlib):
    reqs = _requests(8, seed=9)
    opts = bmlib.make_opts(bmlib.BM_CF32_3XTF32_IR)
    budget = 150 << 20
    s = bmlib.bm_server_create(0, slots=4, budget_bytes=budget, opts=opts)
    try:
        Xs = [np.zeros_like(r[5], order="F") for r in reqs]
        tickets = [bmlib.bm_server_submit(s, c.kind, c.params4(), N, k0, k1, form, B, X)
                   for (c, N, k0, k1, form, B), X in zip(reqs, Xs)]
        results = [bmlib.bm_server_wait(s, t) for t in tickets]
        st = bmlib.bm_server_stats_get(s)
    finally:
        bmlib.bm_server_destroy(s)
    assert all(r.status == 0 and r.backward_error <= 1e-9 for r in results)
    assert st.max_in_flight_bytes <= budget and st.budget_bytes == budget
    assert st.max_in_flight >= 1 and max(r.bytes for r in results) * st.max_in_flight >= st.max_in_flight_bytes
    s = bmlib.bm_server_create(0, slots=2, budget_bytes=1 << 20, opts=opts)
    try:
        c, N, k0, k1, form, B = reqs[0]
        with pytest.raises(bmlib.BMError) as e:
            bmlib.bm_server_submit(s, c.kind, c.params4(), N, k0, k1, form, B, np.zeros_like(B, order="F"))
        assert e.value.status == bmlib.BM_ENOMEM
    finally:
        bmlib.bm_server_destroy(s)

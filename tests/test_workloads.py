"""The seeded input recipes (no GPU): the benchmark scatterers, the complex Gaussian right-hand
sides, their placement in the two systems, and the serving stream's request distribution."""
import numpy as np
import pytest

import workloads as W


def test_named_workloads_match_their_configurations():
    c = W.CIRCLE_N256
    assert (c.curve.kind, c.curve.p[0], c.N, c.k_out, c.k_in, c.nrhs) == (W.CIRCLE, 1.0, 256, 2.0, 3.0, 1)
    s = W.STAR_N4096
    assert (s.curve.kind, s.curve.params4()) == (W.STAR, (1.0, 0.3, 5.0, 0.0))
    assert (s.N, s.k_out, s.k_in, s.n_plane, s.n_gauss, s.seed, s.angles) == (4096, 20.0, 30.0, 1, 64, 0, (0.0,))
    k = W.KITE_N16384
    assert (k.curve.kind, k.curve.params4()) == (W.KITE, (0.65, 1.5, 0.0, 0.0))
    assert (k.N, k.k_out, k.k_in, k.nrhs) == (16384, 100.0, 150.0, 8)
    t = W.scaled(s, 512)
    assert (t.N, t.curve, t.k_out, t.k_in, t.nrhs, t.seed) == (512, s.curve, s.k_out, s.k_in, s.nrhs, s.seed)


def test_gaussian_columns_are_seeded_standard_complex_normals():
    g = W.gaussian_g(4096, 64, seed=0)
    assert g.shape == (4096, 64) and g.dtype == np.complex128
    assert np.array_equal(g, W.gaussian_g(4096, 64, seed=0))
    assert not np.array_equal(g, W.gaussian_g(4096, 64, seed=1))
    n = g.size
    # N(0, 1/2) + i N(0, 1/2): mean 0, E|z|^2 = 1, Re and Im uncorrelated with equal variance
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 5 / np.sqrt(n)
    assert abs(np.mean(g.real ** 2) - 0.5) < 5 / np.sqrt(n)
    assert abs(np.mean(g.real * g.imag)) < 5 / np.sqrt(n)
    assert abs(np.mean(g * g)) < 5 / np.sqrt(n)      # circular: E z^2 = 0


@pytest.mark.parametrize("form, rows, at", [(W.MIXED, 3, 2), (W.ORDINARY, 2, 0)])
def test_place_rhs_puts_the_data_in_the_scattering_block(form, rows, at):
    N = 37
    g = W.gaussian_g(N, 5, seed=3)
    B = W.place_rhs(g, N, form)
    assert B.shape == (rows * N, 5)
    assert np.array_equal(B[at * N:(at + 1) * N], g)
    rest = np.delete(B, np.s_[at * N:(at + 1) * N], axis=0)
    assert not rest.any()


def test_serving_stream_follows_the_request_distribution():
    reqs = W.serving_stream(2000, seed=0)
    assert len(reqs) == 2000
    assert reqs == W.serving_stream(2000, seed=0)
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # unit-rate Poisson arrivals: exponential gaps, mean 1 and standard deviation 1
    assert abs(gaps.mean() - 1.0) < 0.1 and abs(gaps.std() - 1.0) < 0.1
    assert set(r["N"] for r in reqs) == {256, 512, 1024, 2048, 4096, 8192}
    lobes = [r["curve"].p[2] for r in reqs]
    assert set(lobes) == {3.0, 4.0, 5.0, 6.0, 7.0, 8.0}
    amp = np.array([r["curve"].p[1] for r in reqs])
    assert amp.min() >= 0.1 and amp.max() <= 0.3 and abs(amp.mean() - 0.2) < 0.01
    assert all(r["curve"].kind == W.STAR and r["curve"].p[0] == 1.0 for r in reqs)
    k = np.array([r["k_out"] for r in reqs])
    assert k.real.min() >= 2.0 and k.real.max() <= 40.0 and k.imag.min() >= -0.5 and k.imag.max() <= 0.0
    assert all(r["k_in"] == 1.5 * r["k_out"] for r in reqs)
    nrhs = [r["nrhs"] for r in reqs]
    assert min(nrhs) == 1 and max(nrhs) == 64

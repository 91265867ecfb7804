"""GPU parity for the contour eigenvalue solver (bm_ssm, block Sakurai-Sugiura, §5.3 sec:ssm).

* The paper's check (circle radius 0.5, eps1 = 4, double eigenvalue at the zero of H_2^(1) from
  Table tb:ssm_eigenvalues): the device result equals the oracle's on the same probe vectors
  (1e-9 FP64, 1e-7 after 3xTF32 + refinement: the solves carry a 1e-9 backward error) for both
  formulations, and sits within the discretisation error of the tabulated zero.
* The contour-batch workload at full size (ellipse 1.0/0.6, N = 1024, k_in = 1.5 k_out, circle of
  centre 5 and radius 0.5, 32 points, 16 probes, 4 moments): rank, the count inside the contour
  (none), the leading singular values and the eigenvalue estimates against the oracle's values
  stored by tests/golden/make_ssm_golden.py.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import ssm

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _zero(n):
    for line in open(os.path.join(GOLD, "hankel_zeros.txt")):
        f = line.split()
        if f and f[0] == str(n) and f[1] == "reference_doring":
            return complex(float(f[2]), float(f[3]))
    raise KeyError(n)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("prec", [0, 2])
def test_ssm_hankel_zero_matches_oracle(bmlib, form, prec):
    N, target = 128, _zero(2)
    nsys = 3 * N if form == 0 else 2 * N
    V = np.asfortranarray(W.gaussian_full(nsys, 4, 3))
    curve = W.circle(0.5)
    # the true singular values fall from 1 to 0.3 and then to the solver's noise: cut at 1e-6
    om, sig, info = bmlib.bm_ssm(0, curve.kind, curve.params4(), N, form, bmlib.make_opts(prec), target, 0.05, 32, 4,
                                 2.0, V, rank_tol=1e-6)
    inside_ref, _, s_ref = ssm.ssm(curve, N, 2.0, form, target, 0.05, 32, 4, V, 1e-6)
    assert info.n_inside == 2 == inside_ref.size
    got = np.sort_complex(om[:info.n_inside])
    tol = 1e-9 if prec == 0 else 1e-7
    assert np.abs(got - inside_ref).max() < tol, (got, inside_ref)
    assert np.abs(got - target).max() < 5e-6
    assert np.abs(sig[:2] - s_ref[:2]).max() < (1e-10 if prec == 0 else 1e-7) * s_ref[0]
    if prec != 0:
        assert info.max_backward_error <= 1e-9


def _golden():
    g = {"sigma": [], "omega": []}
    for line in open(os.path.join(GOLD, "ssm_ellipse_n1024.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] in ("rank", "n_inside"):
            g[f[0]] = int(f[1])
        elif f[0] == "sigma":
            g["sigma"].append(float(f[1]))
        else:
            g["omega"].append(complex(float(f[1]), float(f[2])))
    return g


@pytest.mark.parametrize("prec,resid", [(2, 2), (2, 4), (0, 2)])
def test_ssm_contour_batch_n1024(bmlib, prec, resid):
    g = _golden()
    N, L = 1024, 16
    V = np.asfortranarray(W.gaussian_full(3 * N, L, 0))
    curve = W.ellipse(1.0, 0.6)
    # The contour runs ~0.25 from resonances, where T(z) is ill-conditioned, and the moments' noise
    # must stay below the 1e-6 rank cut: FP32 factors then need every residual formed afresh to
    # FP64 accuracy (in FP64, resid 2, or from nine-digit tensor-core products, resid 4), refined
    # to about the FP64 solve's own backward error (equal accuracy with the FP64 path).
    opts = bmlib.make_opts(prec, refine_tol=1e-15, residual=resid)
    om, sig, info = bmlib.bm_ssm(0, curve.kind, curve.params4(), N, 0, opts, 5.0, 0.5, 32, 4, 1.5, V, rank_tol=1e-6)
    assert info.rank == g["rank"] and info.n_inside == g["n_inside"] == 0
    s = np.array(g["sigma"])
    r = g["rank"]
    # the singular values above the cut are determined to the moments' accuracy
    assert np.abs(sig[:r] - s[:r]).max() < 1e-6 * s[0]
    assert sig[r] < 1e-6 * sig[0] < sig[r - 1]
    # eigenvalue estimates outside the contour are only loosely determined by the moments
    ref = np.sort_complex(np.array(g["omega"]))
    assert np.abs(np.sort_complex(om) - ref).max() < 2e-3 * np.abs(ref).max()


def test_ssm_batches_and_cluster_sizes_agree(bmlib):
    # the same contour in batches of 5 points (the last one ragged) and of all 16, with a fixed and an
    # autotuned panel cluster: every result agrees (each point's solve is deterministic and the
    # moments sum the points in a fixed order)
    N, target = 128, _zero(2)
    V = np.asfortranarray(W.gaussian_full(3 * N, 4, 3))
    curve = W.circle(0.5)
    out = []
    for batch, cl in ((16, 0), (5, 4), (16, 16)):
        om, sig, info = bmlib.bm_ssm(0, curve.kind, curve.params4(), N, 0, bmlib.make_opts(2), target, 0.05, 16, 4,
                                     2.0, V, rank_tol=1e-6, batch=batch, panel_cluster=cl)
        assert info.batch == batch and info.n_inside == 2
        assert info.panel_cluster in ((16, 8, 4) if cl == 0 else (cl,))
        if cl == 0:
            assert all(t > 0 for t in info.tune_ms)
        out.append((np.sort_complex(om[:2]), sig[:2].copy()))
    for om, sig in out[1:]:
        assert np.abs(om - out[0][0]).max() < 1e-9
        assert np.abs(sig - out[0][1]).max() < 1e-9 * out[0][1][0]

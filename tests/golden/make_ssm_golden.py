"""Writes ssm_ellipse_n1024.txt: the oracle's block Sakurai-Sugiura result for the contour-batch
workload (ellipse semi-axes 1.0 / 0.6, N = 1024, mixed system, k_in = 1.5 k_out, circle of centre 5
and radius 0.5 with 32 trapezoid points, 16 seeded Gaussian probe columns (seed 0), 4 moments,
rank cut 1e-6).  Calls only oracle/ and workloads.py.  Usage: python tests/golden/make_ssm_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ssm  # noqa: E402

N, P, M, L, SEED, TOL = 1024, 32, 4, 16, 0, 1e-6
CENTER, RADIUS, RATIO = 5.0, 0.5, 1.5


def main():
    V = W.gaussian_full(3 * N, L, SEED)
    mu = ssm.moments(ssm.bie_solver(W.ellipse(1.0, 0.6), N, RATIO, W.MIXED), CENTER, RADIUS, P, M, V)
    inside, omega, s = ssm.hankel_eigs(mu, CENTER, RADIUS, TOL)
    r = int(np.sum(s > TOL * s[0]))
    with open(os.path.join(HERE, "ssm_ellipse_n1024.txt"), "w") as f:
        f.write("# oracle block Sakurai-Sugiura, ellipse 1.0/0.6, N=1024, mixed, k_in=1.5 k_out, circle centre 5\n")
        f.write("# radius 0.5, 32 points, 16 Gaussian probes (seed 0), M=4, rank cut 1e-6; written by make_ssm_golden.py\n")
        f.write(f"rank {r}\n")
        f.write(f"n_inside {len(inside)}\n")
        for v in s[:16]:
            f.write(f"sigma {v:.17e}\n")
        for z in np.sort_complex(omega):
            f.write(f"omega {z.real:.17e} {z.imag:.17e}\n")


if __name__ == "__main__":
    main()

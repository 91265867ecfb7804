"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module holds *inputs only*: curve descriptions (kind + parameters), node
counts, wavenumbers, and the random right-hand sides a workload draws.  It
contains none of the method's arithmetic (no geometry evaluation, no kernels,
no Hankel functions, no linear algebra), so that the oracle and the CUDA path
can both consume it without sharing any computation.

Curve kinds and their parameter vectors ``p`` (all parametrised over
t in [0, 2*pi), counter-clockwise):

* ``CIRCLE``  : p = (R, cx, cy)             x = (cx + R cos t, cy + R sin t)
* ``ELLIPSE`` : p = (a, b)                   x = (a cos t, b sin t)
* ``STAR``    : p = (r0, amp, lobes)         r(t) = r0 + amp cos(lobes t), x = r(t)(cos t, sin t)
* ``KITE``    : p = (c, b)                   x = (cos t + c cos 2t - c, b sin t)

The enum values match ``bm_curve_kind`` in ``include/bm.h``.

Workloads follow the scatterers of §5.1 (circle, plane wave e^{i k0 x1}) and
the shapes the benchmark configurations name (star, ellipse, kite).
Material reading: eps0 = 1, omega = k_out, eps1 = (k_in / k_out)^2, beta = i / k_out
(the paper leaves beta free apart from Im beta != 0).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

CIRCLE, ELLIPSE, STAR, KITE, USER = 0, 1, 2, 3, 4
MIXED, ORDINARY = 0, 1
FP64, CF32_TF32_IR, CF32_3XTF32_IR = 0, 1, 2


@dataclass(frozen=True)
class Curve:
    kind: int
    p: tuple = ()

    def params4(self) -> tuple:
        q = list(self.p) + [0.0] * (4 - len(self.p))
        return tuple(float(v) for v in q[:4])


def circle(R=1.0, cx=0.0, cy=0.0) -> Curve:
    return Curve(CIRCLE, (R, cx, cy))


def ellipse(a=1.0, b=0.6) -> Curve:
    return Curve(ELLIPSE, (a, b))


def star(r0=1.0, amp=0.3, lobes=5) -> Curve:
    return Curve(STAR, (r0, amp, float(lobes)))


def kite(c=0.65, b=1.5) -> Curve:
    return Curve(KITE, (c, b))


@dataclass(frozen=True)
class Workload:
    """One scattering solve: a curve, N nodes, two wavenumbers and the RHS recipe."""
    name: str
    curve: Curve
    N: int
    k_out: complex
    k_in: complex
    n_plane: int = 1          # plane-wave RHS columns (incidence angles below)
    n_gauss: int = 0          # seeded complex Gaussian RHS columns
    seed: int = 0
    angles: tuple = (0.0,)    # plane-wave incidence angles (radians)
    extra: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return self.n_plane + self.n_gauss


# Small circle case of §5.1 shape (checked against the Bessel-series solution).
CIRCLE_N256 = Workload("circle R=1 N=256 k=2/3", circle(1.0), 256, 2.0, 3.0)
# Star r = 1 + 0.3 cos 5t, N = 4096, 1 plane wave + 64 Gaussian RHS.
STAR_N4096 = Workload("star 1+0.3cos5t N=4096 k=20/30 nrhs=65", star(1.0, 0.3, 5), 4096, 20.0, 30.0,
                      n_plane=1, n_gauss=64, seed=0)
# Kite N = 16384, 1 plane wave + 7 Gaussian RHS.
KITE_N16384 = Workload("kite N=16384 k=100/150 nrhs=8", kite(), 16384, 100.0, 150.0,
                       n_plane=1, n_gauss=7, seed=0)


def scaled(w: Workload, N: int, n_gauss: int | None = None) -> Workload:
    """The same scatterer and wavenumbers at another node count (for oracle-sized cases)."""
    return Workload(w.name + f" (N={N})", w.curve, N, w.k_out, w.k_in, w.n_plane,
                    w.n_gauss if n_gauss is None else n_gauss, w.seed, w.angles, dict(w.extra))


def gaussian_g(N: int, ncols: int, seed: int = 0) -> np.ndarray:
    """Complex Gaussian columns (N(0,1/2) + i N(0,1/2)), numpy PCG64(seed), shape (N, ncols)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.normal(0.0, np.sqrt(0.5), size=(ncols, N))
    im = rng.normal(0.0, np.sqrt(0.5), size=(ncols, N))
    return np.ascontiguousarray((re + 1j * im).T)


def gaussian_full(rows: int, ncols: int, seed: int = 1) -> np.ndarray:
    """A full complex Gaussian block (every system row), used to exercise arbitrary right-hand sides."""
    return gaussian_g(rows, ncols, seed)


def place_rhs(g: np.ndarray, N: int, formulation: int) -> np.ndarray:
    """Place an N-long data column g into the system RHS: (0, 0, g) mixed, (g, 0) ordinary."""
    nrhs = g.shape[1]
    if formulation == MIXED:
        B = np.zeros((3 * N, nrhs), dtype=np.complex128)
        B[2 * N:] = g
    else:
        B = np.zeros((2 * N, nrhs), dtype=np.complex128)
        B[:N] = g
    return B


def serving_stream(n_requests: int = 2000, seed: int = 0):
    """Requests of the serving stream: Poisson arrivals (unit rate; scale by lambda), star curves
    with lobes U{3..8} and amplitude U[0.1, 0.3], N in {256..8192}, complex k_out, nrhs U{1..64}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0, size=n_requests)
    out = []
    t = 0.0
    Ns = [256, 512, 1024, 2048, 4096, 8192]
    for r in range(n_requests):
        t += gaps[r]
        lobes = int(rng.integers(3, 9))
        amp = float(rng.uniform(0.1, 0.3))
        N = int(Ns[rng.integers(0, len(Ns))])
        k = complex(rng.uniform(2.0, 40.0), rng.uniform(-0.5, 0.0))
        nrhs = int(rng.integers(1, 65))
        out.append(dict(t=t, curve=star(1.0, amp, lobes), N=N, k_out=k, k_in=1.5 * k, nrhs=nrhs))
    return out

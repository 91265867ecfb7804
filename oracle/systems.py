"""Oracle discrete systems: the 3N mixed system and the 2N ordinary system (test infrastructure only).

* Mixed (direct-indirect) system, Eq. dis_mixedBM (§4) in the block names of
  Theorem thm:LU (§4.1):
      [ I    0    M13 ] [u]   [0 ]      M13 = -S_{k1}
      [ 0    I    M23 ] [q] = [0 ]      M23 = -(1/eps1)(D*_{k1} + I/2)
      [ M31  M32  0   ] [phi] [b3]      M31 = D_{k0} - I/2 + beta N_{k0}
                                        M32 = -eps0 (S_{k0} + beta (D*_{k0} + I/2))
                                        b3  = -u_in - beta q_in
* Ordinary system, Eq. dis_BM (§4):
      [ M31            M32          ] [u]   [b3]
      [ D_{k1} + I/2   -eps1 S_{k1} ] [q] = [0 ]
  Reading: Eq. dis_BM prints -S_{k1} in the (2,2) block; the interior Green
  identity with du1/dnu = eps1 q (Eq. problem) gives -eps1 S_{k1}, and only that
  reading converges to the Bessel-series solution when eps1 != 1.  The literal
  form is kept behind ``literal_ordinary=True`` to demonstrate this.

Material reading (§2.1 k_i = omega sqrt(eps_i)): eps0 = 1, omega = k_out,
eps1 = (k_in/k_out)^2; Burton-Miller constant beta = i/k_out (§3.1 only asks Im beta != 0).
Incident plane wave (Table tb:lu_parameters): u_in = exp(i k0 dhat.x), q_in = du_in/dnu.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

import workloads as W
from .geometry import Geometry, nodes
from .operators import layer_entries, layer_operators


@dataclass
class Params:
    k0: complex
    k1: complex
    eps0: complex
    eps1: complex
    beta: complex


def default_params(k_out, k_in, eps0=1.0, eps1=None, beta=None) -> Params:
    k0, k1 = complex(k_out), complex(k_in)
    if eps1 is None:
        eps1 = eps0 * (k1 / k0) ** 2
    if beta is None:
        beta = 1j / k0
    return Params(k0, k1, complex(eps0), complex(eps1), complex(beta))


def mixed_blocks(g: Geometry, P: Params, zeta_p: int = 0):
    """M13, M23, M31, M32 of Theorem thm:LU (each N x N complex); zeta_p selects the quadrature
    (0: the one-point rule of §4, p > 0: order 2p + 3, see ``oracle.zeta``)."""
    I = np.eye(g.N)
    o0 = layer_operators(g, P.k0, zeta_p)
    o1 = layer_operators(g, P.k1, zeta_p)
    M13 = -o1["S"]
    M23 = -(o1["Ds"] + 0.5 * I) / P.eps1
    M31 = o0["D"] - 0.5 * I + P.beta * o0["N"]
    M32 = -P.eps0 * (o0["S"] + P.beta * (o0["Ds"] + 0.5 * I))
    return M13, M23, M31, M32


def mixed_matrix(blocks) -> np.ndarray:
    """The full 3N x 3N matrix of Eq. dis_mixedBM with its identity and zero blocks."""
    M13, M23, M31, M32 = blocks
    N = M13.shape[0]
    A = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    A[:N, :N] = np.eye(N)
    A[N:2 * N, N:2 * N] = np.eye(N)
    A[:N, 2 * N:] = M13
    A[N:2 * N, 2 * N:] = M23
    A[2 * N:, :N] = M31
    A[2 * N:, N:2 * N] = M32
    return A


def ordinary_matrix(g: Geometry, P: Params, literal_ordinary: bool = False, zeta_p: int = 0) -> np.ndarray:
    """The 2N x 2N matrix of Eq. dis_BM (with the eps1 reading of its (2,2) block)."""
    N = g.N
    I = np.eye(N)
    o0 = layer_operators(g, P.k0, zeta_p)
    o1 = layer_operators(g, P.k1, zeta_p)
    A = np.zeros((2 * N, 2 * N), dtype=np.complex128)
    A[:N, :N] = o0["D"] - 0.5 * I + P.beta * o0["N"]
    A[:N, N:] = -P.eps0 * (o0["S"] + P.beta * (o0["Ds"] + 0.5 * I))
    A[N:, :N] = o1["D"] + 0.5 * I
    A[N:, N:] = -(1.0 if literal_ordinary else P.eps1) * o1["S"]
    return A


def _row_ops(g: Geometry, k: complex, i: int) -> dict:
    """Row i of S_k, D_k, D*_k, N_k (all N columns), entry by entry."""
    J = np.arange(g.N)
    return layer_entries(g, k, np.full(g.N, i), J)


def mixed_rows(g: Geometry, P: Params, rows) -> np.ndarray:
    """Selected rows (indices in 0..3N-1) of the 3N mixed matrix of Eq. dis_mixedBM, each built
    from its own operator entries - for checks at sizes where the full matrix is too large."""
    N = g.N
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((rows.size, 3 * N), dtype=np.complex128)
    for a, i in enumerate(rows):
        blk, ii = divmod(int(i), N)
        e = np.zeros(N)
        e[ii] = 1.0
        if blk == 0:    # [I 0 M13]
            out[a, ii] = 1.0
            out[a, 2 * N:] = -_row_ops(g, P.k1, ii)["S"]
        elif blk == 1:  # [0 I M23]
            out[a, N + ii] = 1.0
            out[a, 2 * N:] = -(_row_ops(g, P.k1, ii)["Ds"] + 0.5 * e) / P.eps1
        else:           # [M31 M32 0]
            o0 = _row_ops(g, P.k0, ii)
            out[a, :N] = o0["D"] - 0.5 * e + P.beta * o0["N"]
            out[a, N:2 * N] = -P.eps0 * (o0["S"] + P.beta * (o0["Ds"] + 0.5 * e))
    return out


def ordinary_rows(g: Geometry, P: Params, rows) -> np.ndarray:
    """Selected rows (indices in 0..2N-1) of the 2N ordinary matrix of Eq. dis_BM (eps1 reading)."""
    N = g.N
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((rows.size, 2 * N), dtype=np.complex128)
    for a, i in enumerate(rows):
        blk, ii = divmod(int(i), N)
        e = np.zeros(N)
        e[ii] = 1.0
        if blk == 0:
            o0 = _row_ops(g, P.k0, ii)
            out[a, :N] = o0["D"] - 0.5 * e + P.beta * o0["N"]
            out[a, N:] = -P.eps0 * (o0["S"] + P.beta * (o0["Ds"] + 0.5 * e))
        else:
            o1 = _row_ops(g, P.k1, ii)
            out[a, :N] = o1["D"] + 0.5 * e
            out[a, N:] = -P.eps1 * o1["S"]
    return out


def incident(g: Geometry, k0: complex, angle: float):
    """Plane wave u_in = exp(i k0 dhat.x) and q_in = du_in/dnu = i k0 (dhat.nu) u_in at the nodes."""
    dh = np.array([np.cos(angle), np.sin(angle)])
    u = np.exp(1j * k0 * (g.x @ dh))
    q = 1j * k0 * (g.nu @ dh) * u
    return u, q


def rhs_plane_wave(g: Geometry, P: Params, angles, formulation: int) -> np.ndarray:
    """System right-hand sides for plane waves: b3 = -u_in - beta q_in placed as (0,0,b3) or (b3,0)."""
    cols = []
    for a in angles:
        u, q = incident(g, P.k0, a)
        cols.append(-u - P.beta * q)
    g3 = np.stack(cols, 1)
    return W.place_rhs(g3, g.N, formulation)


def build(w: W.Workload, formulation: int):
    """Convenience: geometry, params and the assembled operator for a workload."""
    g = nodes(w.curve, w.N)
    P = default_params(w.k_out, w.k_in)
    if formulation == W.MIXED:
        return g, P, mixed_blocks(g, P)
    return g, P, ordinary_matrix(g, P)

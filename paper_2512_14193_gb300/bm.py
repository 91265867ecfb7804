"""Python binding of the C ABI in include/bm.h (ctypes; argument marshalling only).

Every function has the name of its C entry point and forwards to libbm.so; all computation
happens in the library's CUDA kernels.  There is no fallback: if libbm.so is missing or a call
fails, a BMError is raised.

Arrays: complex matrices are column-major complex128.  Host arrays are numpy arrays
(Fortran order); device arrays are torch complex128 CUDA tensors whose first dimension is
contiguous (``t.stride(0) == 1``), e.g. ``torch.empty((ncols, rows), dtype=torch.complex128,
device='cuda').t()``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbm.so")

BM_OK, BM_EINVAL, BM_ENOMEM, BM_ESINGULAR, BM_ENOTCONV, BM_ENONFINITE, BM_ETIMEOUT, BM_ESTATE, BM_ECUDA = range(9)
BM_MIXED, BM_ORDINARY = 0, 1
BM_FP64, BM_CF32_TF32_IR, BM_CF32_3XTF32_IR = 0, 1, 2
BM_CURVE_CIRCLE, BM_CURVE_ELLIPSE, BM_CURVE_STAR, BM_CURVE_KITE, BM_CURVE_USER = range(5)
BM_PROBE_SCHUR, BM_PROBE_RESIDUAL = 0, 1
BM_RESID_TC_UPDATE, BM_RESID_FP64_UPDATE, BM_RESID_FP64_ALL, BM_RESID_DF_UPDATE, BM_RESID_TC_ALL = 0, 1, 2, 3, 4
BM_FAR_FIELD_STATIC_MAX_ANGLES = 8192


class bm_c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class bm_curve(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 4), ("user", C.POINTER(C.c_double))]


class bm_opts(C.Structure):
    _fields_ = [("eps0", C.c_double), ("eps1", bm_c64), ("beta", bm_c64), ("eps_set", C.c_int),
                ("beta_set", C.c_int), ("prec", C.c_int), ("refine_tol", C.c_double), ("refine_maxit", C.c_int),
                ("nb", C.c_int), ("refine_residual", C.c_int), ("zeta_p", C.c_int), ("eager", C.c_int),
                ("panel_cluster_max", C.c_int), ("panel_kernel", C.c_int), ("test_wait_timeout", C.c_int)]


class bm_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("backward_error", C.c_double), ("t_solve_ms", C.c_double),
                ("t_residual_ms", C.c_double)]


class bm_ssm_opts(C.Structure):
    _fields_ = [("center", bm_c64), ("radius", C.c_double), ("npoints", C.c_int), ("nmoments", C.c_int),
                ("k_ratio", bm_c64), ("rank_tol", C.c_double), ("workers", C.c_int), ("batch", C.c_int),
                ("panel_cluster", C.c_int)]


class bm_ssm_info(C.Structure):
    _fields_ = [("rank", C.c_int), ("n_inside", C.c_int), ("max_iterations", C.c_int),
                ("max_backward_error", C.c_double), ("t_total_ms", C.c_double), ("t_points_ms", C.c_double),
                ("t_assemble_ms", C.c_double), ("t_factor_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("batch", C.c_int), ("panel_cluster", C.c_int), ("tune_ms", C.c_double * 3)]


class bm_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("opts", bm_opts)]


class bm_request(C.Structure):
    _fields_ = [("curve", bm_curve), ("N", C.c_int), ("k_out", bm_c64), ("k_in", bm_c64), ("formulation", C.c_int),
                ("nrhs", C.c_int), ("B", C.c_void_p), ("ldb", C.c_int), ("X", C.c_void_p), ("ldx", C.c_int)]


class bm_result(C.Structure):
    _fields_ = [("status", C.c_int), ("slot", C.c_int), ("iterations", C.c_int), ("backward_error", C.c_double),
                ("t_queue_ms", C.c_double), ("t_service_ms", C.c_double), ("bytes", C.c_size_t)]


class bm_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("launches", C.c_int), ("ms", C.c_double)]


class bm_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_ulonglong), ("completed", C.c_ulonglong), ("max_in_flight_bytes", C.c_size_t),
                ("max_in_flight", C.c_int), ("budget_bytes", C.c_size_t)]


class BMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        L = lib()
        super().__init__(f"{where}: {L.bm_strerror(status).decode()} ({L.bm_last_error().decode()})")


_lib = None


def lib():
    """Load libbm.so (built in-tree by paper_2512_14193_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2512_14193_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    L.bm_create.argtypes = [C.POINTER(P), I, P, S]
    L.bm_assemble.argtypes = [P, C.POINTER(bm_curve), I, bm_c64, bm_c64, I, C.POINTER(bm_opts)]
    L.bm_factor.argtypes = [P, C.POINTER(I)]
    L.bm_rhs_plane_wave.argtypes = [P, C.POINTER(D), I, P, I, I]
    L.bm_solve.argtypes = [P, I, P, I, P, I, I, C.POINTER(bm_solve_info)]
    L.bm_solve_block.argtypes = [P, I, P, I, I, P, I, I, P, I, P, I, I, C.POINTER(bm_solve_info)]
    L.bm_far_field.argtypes = [P, P, I, I, C.POINTER(D), I, P, I, I]
    L.bm_far_field_static.argtypes = [P, P, I, I, C.POINTER(D), I, P, I]
    L.bm_copy_block.argtypes = [P, I, P, I, I]
    L.bm_server_create.argtypes = [C.POINTER(P), I, C.POINTER(bm_server_opts)]
    L.bm_server_submit.argtypes = [P, C.POINTER(bm_request), C.POINTER(C.c_ulonglong)]
    L.bm_server_wait.argtypes = [P, C.c_ulonglong, C.POINTER(bm_result)]
    L.bm_server_stats_get.argtypes = [P, C.POINTER(bm_server_stats)]
    L.bm_server_destroy.argtypes = [P]
    L.bm_ssm.argtypes = [I, C.POINTER(bm_curve), I, I, C.POINTER(bm_opts), C.POINTER(bm_ssm_opts), P, I, I, P, I,
                         C.POINTER(D), C.POINTER(bm_ssm_info)]
    L.bm_hankel01.argtypes = [P, P, I, P, P, I]
    L.bm_ssm_release.argtypes = [I]
    L.bm_zeta_weights.argtypes = [I, C.POINTER(D), C.POINTER(D)]
    L.bm_hankel_anchor_table.argtypes = [C.POINTER(D), I, C.POINTER(I), C.POINTER(I), C.POINTER(D), C.POINTER(D),
                                         C.POINTER(D)]
    L.bm_hankel_taylor_table.argtypes = [C.POINTER(D), I, C.POINTER(I)]
    L.bm_f32_convert.argtypes = [P, P, I, P]
    L.bm_memory.argtypes = [P, C.POINTER(S), C.POINTER(S)]
    L.bm_kernel_launches.argtypes = [P, C.POINTER(C.c_ulonglong)]
    L.bm_enqueue_probe.argtypes = [P, I, I]
    L.bm_profile.argtypes = [P, I, P, I, P, I, I, C.POINTER(bm_kernel_time), I, C.POINTER(I)]
    L.bm_destroy.argtypes = [P]
    L.bm_strerror.argtypes = [I]
    L.bm_strerror.restype = C.c_char_p
    L.bm_last_error.argtypes = []
    L.bm_last_error.restype = C.c_char_p
    for name in ("bm_create", "bm_assemble", "bm_factor", "bm_rhs_plane_wave", "bm_solve", "bm_solve_block",
                 "bm_far_field",
                 "bm_far_field_static", "bm_ssm", "bm_server_create", "bm_server_submit", "bm_server_wait",
                 "bm_server_stats_get", "bm_server_destroy",
                 "bm_copy_block", "bm_hankel01", "bm_f32_convert", "bm_hankel_anchor_table", "bm_hankel_taylor_table",
                 "bm_zeta_weights",
                 "bm_memory",
                 "bm_destroy",
                 "bm_kernel_launches", "bm_enqueue_probe", "bm_profile", "bm_ssm_release"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st: int, where: str, ok=(BM_OK,)):
    if st not in ok:
        raise BMError(st, where)
    return st


# rows of the assembled system per handle (3N mixed, 2N ordinary), for the shape checks below: the
# library sees leading dimensions only, so an array with too few rows or columns must be caught here
_nsys = {}
# order of the blocks bm_copy_block copies per handle (N mixed, 2N ordinary)
_blk = {}
# host arrays of queued serving requests, by (server, ticket), until the request is collected
_in_flight = {}


def _hkey(h) -> int:
    return int(h.value) if isinstance(h, C.c_void_p) and h.value is not None else id(h)


def _need(cond: bool, msg: str) -> None:
    if not cond:
        raise ValueError(msg)


def _c64(z) -> bm_c64:
    z = complex(z)
    return bm_c64(z.real, z.imag)


# --------------------------------------------------------------------------------------------
# array marshalling: (pointer, leading dimension, ncols, on_device)
# --------------------------------------------------------------------------------------------
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _colmajor(a, rows_min: int, writable: bool):
    if _is_torch(a):
        import torch
        if a.dtype != torch.complex128:
            raise TypeError("torch arrays must be complex128")
        if a.dim() == 1:
            a = a.unsqueeze(1)
        if a.stride(0) != 1:
            raise ValueError("torch arrays must be column-major (stride(0) == 1)")
        ld = a.stride(1) if a.shape[1] > 1 else max(a.shape[0], 1)
        if a.is_cuda:
            torch.cuda.current_stream(a.device).synchronize()
        # CPU tensors (e.g. pinned host buffers) are passed as host pointers
        return C.c_void_p(a.data_ptr()), int(ld), int(a.shape[1]), 1 if a.is_cuda else 0, a
    arr = np.asarray(a)
    if arr.ndim == 1:
        arr = arr.reshape(-1, 1, order="F")
    if arr.dtype != np.complex128 or not arr.flags.f_contiguous:
        if writable:
            raise ValueError("host output arrays must be Fortran-ordered complex128")
        arr = np.asfortranarray(arr, dtype=np.complex128)
    return C.c_void_p(arr.ctypes.data), int(arr.shape[0]), int(arr.shape[1]), 0, arr


# --------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------------------------
def bm_create(device: int = 0, stream: int | None = None, budget_bytes: int = 0):
    h = C.c_void_p()
    _check(lib().bm_create(C.byref(h), int(device), C.c_void_p(stream or 0), int(budget_bytes)), "bm_create")
    return h


def bm_destroy(h) -> None:
    _nsys.pop(_hkey(h), None)
    _blk.pop(_hkey(h), None)
    _check(lib().bm_destroy(h), "bm_destroy")


def make_opts(prec: int = BM_FP64, eps0: float = 1.0, eps1=None, beta=None, refine_tol: float = 1e-9,
              refine_maxit: int = 30, nb: int = 0, residual: int = 0, zeta_p: int = 0, eager: bool = False,
              panel_cluster_max: int = 0, panel_kernel: int = 0, test_wait_timeout: int = 0) -> bm_opts:
    o = bm_opts()
    o.zeta_p = int(zeta_p)
    o.eager = int(bool(eager))
    o.panel_cluster_max = int(panel_cluster_max)
    o.panel_kernel = int(panel_kernel)
    o.test_wait_timeout = int(test_wait_timeout)
    o.eps0 = float(eps0)
    o.prec = int(prec)
    o.refine_tol = float(refine_tol)
    o.refine_maxit = int(refine_maxit)
    o.nb = int(nb)
    o.refine_residual = int(residual)
    if eps1 is not None:
        o.eps1 = _c64(eps1)
        o.eps_set = 1
    if beta is not None:
        o.beta = _c64(beta)
        o.beta_set = 1
    return o


def bm_assemble(h, kind: int, params, N: int, k_out, k_in, formulation: int = BM_MIXED, opts: bm_opts | None = None,
                user: np.ndarray | None = None) -> None:
    cv = bm_curve()
    cv.kind = int(kind)
    p = list(params) + [0.0] * (4 - len(params))
    for i in range(4):
        cv.p[i] = float(p[i])
    keep = None
    if user is not None:
        keep = np.ascontiguousarray(user, dtype=np.float64)
        cv.user = keep.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib().bm_assemble(h, C.byref(cv), int(N), _c64(k_out), _c64(k_in), int(formulation),
                             C.byref(opts) if opts is not None else None), "bm_assemble")
    _nsys[_hkey(h)] = (3 if int(formulation) == BM_MIXED else 2) * int(N)
    _blk[_hkey(h)] = (1 if int(formulation) == BM_MIXED else 2) * int(N)


def bm_factor(h) -> int:
    info = C.c_int(0)
    st = lib().bm_factor(h, C.byref(info))
    _check(st, "bm_factor", ok=(BM_OK, BM_ESINGULAR))
    return int(info.value)


def bm_rhs_plane_wave(h, angles, B) -> None:
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    ptr, ld, ncols, dev, _keep = _colmajor(B, 0, writable=True)
    _need(ncols >= ang.size, "B needs a column per incidence angle")
    _need(_keep.shape[0] >= _nsys.get(_hkey(h), 0), "B has fewer rows than the system")
    _check(lib().bm_rhs_plane_wave(h, ang.ctypes.data_as(C.POINTER(C.c_double)), int(ang.size), ptr, ld, dev),
           "bm_rhs_plane_wave")


def bm_solve(h, B, X, raise_on_notconv: bool = True) -> bm_solve_info:
    pb, ldb, nb, devb, _kb = _colmajor(B, 0, writable=False)
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=True)
    if devb != devx or nb != nx:
        raise ValueError("B and X must live on the same side and have the same number of columns")
    ns = _nsys.get(_hkey(h), 0)
    _need(_kb.shape[0] >= ns and _kx.shape[0] >= ns, "B and X need at least the system's rows")
    info = bm_solve_info()
    st = lib().bm_solve(h, nb, pb, ldb, px, ldx, devb, C.byref(info))
    _check(st, "bm_solve", ok=(BM_OK,) if raise_on_notconv else (BM_OK, BM_ENOTCONV))
    return info


def bm_solve_block(h, B1, B2, B3, X, raise_on_notconv: bool = True) -> bm_solve_info:
    """X = solution for the block-diagonal right-hand side diag(B1, B2, B3) (Corollary lem:block_LU);
    a block may be None (no columns).  All on the host or all CUDA tensors."""
    args, keep, sides = [], [], set()
    for B in (B1, B2, B3):
        if B is None:
            args += [0, None, 1]
            continue
        p, ld, n, dev, k = _colmajor(B, 0, writable=False)
        args += [n, p, ld]
        keep.append(k)
        sides.add(dev)
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=True)
    sides.add(devx)
    _need(nx == sum(a for a in args[0::3]), "X needs one column per column of B1, B2, B3")
    _need(_kx.shape[0] >= _nsys.get(_hkey(h), 0), "X has fewer rows than the system")
    for B, k in zip([b for b in (B1, B2, B3) if b is not None], keep):
        _need(k.shape[0] * 3 >= _nsys.get(_hkey(h), 0), "each block needs N rows")
    if len(sides) != 1:
        raise ValueError("B1, B2, B3 and X must all live on the same side")
    info = bm_solve_info()
    st = lib().bm_solve_block(h, *args, px, ldx, devx, C.byref(info))
    _check(st, "bm_solve_block", ok=(BM_OK,) if raise_on_notconv else (BM_OK, BM_ENOTCONV))
    return info


def _far_field_shapes(h, kx, nx, ku, nu, ang) -> None:
    # the kernel writes M x nrhs values into U and reads nrhs columns of X: U must have a column per
    # column of X and a row per angle, X the system's rows
    _need(nu == nx, f"U has {nu} columns for {nx} solutions")
    _need(ku.shape[0] >= ang.size, f"U has {ku.shape[0]} rows for {ang.size} angles")
    _need(kx.shape[0] >= _nsys.get(_hkey(h), 0), "X has fewer rows than the system")


def bm_far_field(h, X, angles, U) -> None:
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=False)
    pu, ldu, nu, devu, _ku = _colmajor(U, 0, writable=True)
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    _far_field_shapes(h, _kx, nx, _ku, nu, ang)
    _need(devx == devu, "X and U must live on the same side")
    _check(lib().bm_far_field(h, px, ldx, nx, ang.ctypes.data_as(C.POINTER(C.c_double)), int(ang.size), pu, ldu,
                              devx), "bm_far_field")


def bm_far_field_static(h, X, angles, U) -> None:
    """bm_far_field without device allocation; X and U must be CUDA tensors."""
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=False)
    pu, ldu, nu, devu, _ku = _colmajor(U, 0, writable=True)
    if not (devx and devu):
        raise ValueError("bm_far_field_static takes device arrays only")
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    _far_field_shapes(h, _kx, nx, _ku, nu, ang)
    _check(lib().bm_far_field_static(h, px, ldx, nx, ang.ctypes.data_as(C.POINTER(C.c_double)), int(ang.size), pu,
                                     ldu), "bm_far_field_static")


def bm_ssm(device: int, kind: int, params, N: int, formulation: int, opts: bm_opts | None, center, radius: float,
           npoints: int, nmoments: int, k_ratio, V, rank_tol: float = 0.0, workers: int = 0, batch: int = 0,
           panel_cluster: int = 0):
    """Eigenvalues inside a circle (block Sakurai-Sugiura).  V: host (nsys x L) probe columns.
    Returns (omega[r] with the n_inside interior ones first, sigma[L M], bm_ssm_info)."""
    cv = bm_curve()
    cv.kind = int(kind)
    p = list(params) + [0.0] * (4 - len(params))
    for i in range(4):
        cv.p[i] = float(p[i])
    so = bm_ssm_opts()
    so.center = _c64(center)
    so.radius = float(radius)
    so.npoints = int(npoints)
    so.nmoments = int(nmoments)
    so.k_ratio = _c64(k_ratio)
    so.rank_tol = float(rank_tol)
    so.workers = int(workers)
    so.batch = int(batch)
    so.panel_cluster = int(panel_cluster)
    pv, ldv, L, dev, _kv = _colmajor(V, 0, writable=False)
    if dev:
        raise ValueError("bm_ssm takes host probe vectors")
    cap = L * int(nmoments)
    om = np.zeros(cap, dtype=np.complex128)
    sig = np.zeros(cap, dtype=np.float64)
    info = bm_ssm_info()
    _check(lib().bm_ssm(int(device), C.byref(cv), int(N), int(formulation), C.byref(opts) if opts is not None else None,
                        C.byref(so), pv, ldv, L, C.c_void_p(om.ctypes.data), cap,
                        sig.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info)), "bm_ssm")
    return om[:info.rank].copy(), sig, info


def bm_ssm_release(device: int = -1) -> None:
    """Free the contour solver's kept batch of handles and buffers (every device when device < 0)."""
    _check(lib().bm_ssm_release(int(device)), "bm_ssm_release")


def bm_server_create(device: int = 0, slots: int = 4, budget_bytes: int = 0, opts: bm_opts | None = None):
    o = bm_server_opts()
    o.slots = int(slots)
    o.hbm_budget_bytes = int(budget_bytes)
    o.opts = opts if opts is not None else make_opts()
    s = C.c_void_p()
    _check(lib().bm_server_create(C.byref(s), int(device), C.byref(o)), "bm_server_create")
    return s


def bm_server_submit(s, kind: int, params, N: int, k_out, k_in, formulation: int, B: np.ndarray, X: np.ndarray) -> int:
    """Queue a solve; B and X are Fortran-ordered host complex128 arrays.  The binding holds them
    until bm_server_wait returns for the ticket (or bm_server_destroy); X holds the solution then."""
    pb, ldb, nb, devb, _kb = _colmajor(B, 0, writable=False)
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=True)
    if devb or devx or nb != nx:
        raise ValueError("host B and X with the same number of columns")
    if _kb is not B:
        raise ValueError("B must be a Fortran-ordered complex128 array (no temporary copy)")
    r = bm_request()
    r.curve.kind = int(kind)
    p = list(params) + [0.0] * (4 - len(params))
    for i in range(4):
        r.curve.p[i] = float(p[i])
    r.N = int(N)
    r.k_out = _c64(k_out)
    r.k_in = _c64(k_in)
    r.formulation = int(formulation)
    r.nrhs = nb
    r.B, r.ldb, r.X, r.ldx = pb, ldb, px, ldx
    t = C.c_ulonglong(0)
    _check(lib().bm_server_submit(s, C.byref(r), C.byref(t)), "bm_server_submit")
    # the worker reads B and writes X until the request is collected: hold them until then
    _in_flight[(_hkey(s), int(t.value))] = (B, X)
    return int(t.value)


def bm_server_wait(s, ticket: int) -> bm_result:
    res = bm_result()
    st = lib().bm_server_wait(s, C.c_ulonglong(ticket), C.byref(res))
    if st != BM_EINVAL:  # BM_EINVAL: unknown or already collected ticket, nothing was running
        _in_flight.pop((_hkey(s), int(ticket)), None)
    _check(st, "bm_server_wait")
    return res


def bm_server_stats_get(s) -> bm_server_stats:
    st = bm_server_stats()
    _check(lib().bm_server_stats_get(s, C.byref(st)), "bm_server_stats_get")
    return st


def bm_server_destroy(s) -> None:
    st = lib().bm_server_destroy(s)
    key = _hkey(s)
    for k in [k for k in _in_flight if k[0] == key]:  # every request has finished by now
        del _in_flight[k]
    _check(st, "bm_server_destroy")


def bm_copy_block(h, which: int, dst) -> None:
    p, ld, _n, dev, _k = _colmajor(dst, 0, writable=True)
    # the library copies a whole block (N x N mixed, 2N x 2N ordinary) at leading dimension ld
    n = _blk.get(_hkey(h), 0)
    _need(_k.shape[0] >= n and _n >= n, f"dst must hold the {n} x {n} block")
    _check(lib().bm_copy_block(h, int(which), p, ld, dev), "bm_copy_block")


def bm_hankel01(h, z):
    """H0^(1), H1^(1) at complex points z (numpy, evaluated on the device)."""
    zz = np.ascontiguousarray(z, dtype=np.complex128).ravel()
    h0 = np.empty_like(zz)
    h1 = np.empty_like(zz)
    _check(lib().bm_hankel01(h, C.c_void_p(zz.ctypes.data), int(zz.size), C.c_void_p(h0.ctypes.data),
                             C.c_void_p(h1.ctypes.data), 0), "bm_hankel01")
    return h0, h1


def bm_zeta_weights(p: int):
    """(tau[0..p], c2[0..p+1]): the library's high-order zeta correction weights (host only)."""
    tau = np.zeros(p + 1)
    c2 = np.zeros(p + 2)
    _check(lib().bm_zeta_weights(int(p), tau.ctypes.data_as(C.POINTER(C.c_double)),
                                 c2.ctypes.data_as(C.POINTER(C.c_double))), "bm_zeta_weights")
    return tau, c2


def bm_f32_convert(h, x):
    """float32 array: the device's integer FP64 -> FP32 rounding (nearest, ties to even) of x."""
    xs = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    _need(xs.size >= 1, "x must not be empty")
    rn = np.zeros(xs.size, dtype=np.float32)
    _check(lib().bm_f32_convert(h, xs.ctypes.data, int(xs.size), rn.ctypes.data), "bm_f32_convert")
    return rn


def bm_hankel_anchor_table():
    """(table[ny, nx, 2] complex: H0, H1 at anchors, re0, im0, step) - host-built, no GPU needed."""
    nx, ny = C.c_int(), C.c_int()
    re0, im0, step = C.c_double(), C.c_double(), C.c_double()
    L = lib()
    _check(L.bm_hankel_anchor_table(None, 0, C.byref(nx), C.byref(ny), C.byref(re0), C.byref(im0), C.byref(step)),
           "bm_hankel_anchor_table")
    out = np.zeros(4 * nx.value * ny.value, dtype=np.float64)
    _check(L.bm_hankel_anchor_table(out.ctypes.data_as(C.POINTER(C.c_double)), nx.value * ny.value, None, None,
                                    None, None, None), "bm_hankel_anchor_table")
    t = out.view(np.complex128).reshape(ny.value, nx.value, 2)
    return t, re0.value, im0.value, step.value


def bm_hankel_taylor_table():
    """table[ny, nx, nterms] complex: the Taylor coefficients of H0 about every anchor of
    bm_hankel_anchor_table (as the device holds them) - host-built, no GPU needed."""
    T, _re0, _im0, _step = bm_hankel_anchor_table()
    ny, nx = T.shape[0], T.shape[1]
    L = lib()
    K = C.c_int()
    _check(L.bm_hankel_taylor_table(None, 0, C.byref(K)), "bm_hankel_taylor_table")
    out = np.zeros(2 * K.value * nx * ny, dtype=np.float64)
    _check(L.bm_hankel_taylor_table(out.ctypes.data_as(C.POINTER(C.c_double)), nx * ny, None),
           "bm_hankel_taylor_table")
    return out.view(np.complex128).reshape(ny, nx, K.value)


def bm_memory(h):
    held, budget = C.c_size_t(), C.c_size_t()
    _check(lib().bm_memory(h, C.byref(held), C.byref(budget)), "bm_memory")
    return held.value, budget.value


def bm_enqueue_probe(h, which: int, reps: int) -> None:
    _check(lib().bm_enqueue_probe(h, int(which), int(reps)), "bm_enqueue_probe")


def bm_kernel_launches(h) -> int:
    n = C.c_ulonglong(0)
    _check(lib().bm_kernel_launches(h, C.byref(n)), "bm_kernel_launches")
    return int(n.value)


def bm_strerror(status: int) -> str:
    return lib().bm_strerror(int(status)).decode()


def bm_last_error() -> str:
    return lib().bm_last_error().decode()


def bm_profile(h, B, X):
    """Per-kernel device times of one bm_factor + bm_solve(B, X): a list of (name, launches, ms),
    largest first (every kernel launched directly and bracketed by events)."""
    pb, ldb, nb, devb, _kb = _colmajor(B, 0, writable=False)
    px, ldx, nx, devx, _kx = _colmajor(X, 0, writable=True)
    if devb != devx or nb != nx:
        raise ValueError("B and X must live on the same side and have the same number of columns")
    ns = _nsys.get(_hkey(h), 0)
    _need(_kb.shape[0] >= ns and _kx.shape[0] >= ns, "B and X need at least the system's rows")
    cap = 64
    out = (bm_kernel_time * cap)()
    n = C.c_int(0)
    _check(lib().bm_profile(h, nb, pb, ldb, px, ldx, devb, out, cap, C.byref(n)), "bm_profile")
    return [(out[i].name.decode(), int(out[i].launches), float(out[i].ms)) for i in range(min(n.value, cap))]

"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/bm.h declares,
and its host-built Hankel anchor table matches scipy (no GPU needed for any of this)."""
import os
import re

import numpy as np
from scipy import special as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(bmlib):
    import ctypes
    L = ctypes.CDLL(bmlib.LIB_PATH)
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_names_every_status(bmlib):
    for s in range(9):
        assert bmlib.bm_strerror(s).startswith("BM_")


def test_anchor_table_matches_scipy(bmlib):
    T, re0, im0, step = bmlib.bm_hankel_anchor_table()
    ny, nx, _ = T.shape
    iy, ix = np.mgrid[0:ny, 0:nx]
    z = re0 + ix * step + 1j * (im0 + iy * step)
    used = (np.abs(z) >= 2.75) & (np.abs(z) <= 20.25)      # anchors the device Taylor zone can pick
    H0, H1 = sp.hankel1(0, z[used]), sp.hankel1(1, z[used])
    e = np.maximum(np.abs(T[..., 0][used] - H0) / np.abs(H0), np.abs(T[..., 1][used] - H1) / np.abs(H1))
    assert used.sum() > 9000
    assert e.max() < 1e-14


def test_create_without_gpu_reports_cuda_error(bmlib):
    import torch
    if torch.cuda.is_available():
        return
    import ctypes
    h = ctypes.c_void_p()
    st = bmlib.lib().bm_create(ctypes.byref(h), 0, None, 0)
    assert st == bmlib.BM_ECUDA

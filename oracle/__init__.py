"""FP64 CPU oracle for image-centred ray shooting (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never links, loads or calls
it; it shares no code with the CUDA path.  The arithmetic lives in
``icrs_oracle.cpp``; this module compiles it with the host compiler and wraps
its C entry points with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icrs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libicrs_oracle.so")
_lock = threading.Lock()
_lib = None

# Parameter vector layout used by the oracle's C entry points.
PARAM_FIELDS = ("t0", "tE", "u0", "alpha", "rho", "u1", "n_lens",
                "s", "q", "q2", "q3", "s2", "s3", "psi", "u2", "a1", "a2", "a3", "a4",
                "spot_x", "spot_y", "spot_r", "spot_c")
GRID_FIELDS = ("n_r", "n_theta", "n_limb", "n_bins_r", "n_bins_theta",
               "max_iter", "uniform", "delta_c", "margin", "img_tol", "ld_split", "grad_rule", "s_fac")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libicrs_oracle.so`` (g++, -O2, FP64)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


_OMP_PATH = os.path.join(_HERE, "libicrs_oracle_omp.so")
_omp = None


def build_omp(force: bool = False) -> str:
    """The same source compiled with OpenMP: orc_magnification runs its
    epochs on all host cores (the CPU baseline's all-core rate)."""
    with _lock:
        if (not force and os.path.exists(_OMP_PATH)
                and os.path.getmtime(_OMP_PATH) >= os.path.getmtime(_SRC)):
            return _OMP_PATH
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OMP_PATH)
        return _OMP_PATH


def magnification_all_cores(params, t, grid: dict):
    """magnification() through the OpenMP build (threads: OMP_NUM_THREADS,
    else all cores).  Returns (A, status)."""
    global _omp
    if _omp is None:
        build_omp()
        L = ctypes.CDLL(_OMP_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_magnification.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                                        ctypes.POINTER(ctypes.c_uint32)]
        _omp = L
    if isinstance(params, dict):
        params = [params]
    prm = np.stack([param_vector(p) for p in params])
    S = prm.shape[0]
    t = np.asarray(t, dtype=np.float64).reshape(S, -1)
    E = t.shape[1]
    prm, pp = _d(prm); t, tp = _d(t)
    g, gp = _d(grid_vector(grid))
    A = np.zeros((S, E)); st = np.zeros((S, E), dtype=np.uint32)
    _omp.orc_magnification(pp, S, tp, E, gp, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return A, st


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_uint32)
        L.orc_lens.argtypes = [dp, dp, dp, dp]
        L.orc_lens.restype = ctypes.c_int
        L.orc_source_centre.argtypes = [dp, dp, ctypes.c_int, dp, dp]
        L.orc_poly.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, dp, dp]
        L.orc_poly.restype = ctypes.c_int
        L.orc_roots.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
        L.orc_roots.restype = ctypes.c_int
        L.orc_lens_map.argtypes = [dp, dp, dp, ctypes.c_int, dp, dp]
        L.orc_point_source.argtypes = [dp, dp, dp, dp, ctypes.c_int, dp, ip, dp, dp, up]
        L.orc_sectors.argtypes = [dp, ctypes.c_double, dp, dp, ctypes.c_int, up]
        L.orc_sectors.restype = ctypes.c_int
        L.orc_magnification.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp, dp, up]
        L.orc_limb_points.argtypes = [dp, ctypes.c_double, dp, dp]
        L.orc_limb_points.restype = ctypes.c_int
        L.orc_magnification_fwd.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp, dp, dp, up]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def param_vector(p: dict) -> np.ndarray:
    """Flatten a parameter dict into the oracle's 23-slot layout (absent keys: 0)."""
    out = np.zeros(len(PARAM_FIELDS))
    for i, k in enumerate(PARAM_FIELDS):
        out[i] = float(p.get(k, 0.0))
    return out


def grid_vector(g: dict) -> np.ndarray:
    return np.array([float(g.get(k, 0)) for k in GRID_FIELDS])


def lens(p: dict):
    prm, pp = _d(param_vector(p))
    eps = np.zeros(3); ax = np.zeros(3); ay = np.zeros(3)
    _, e_p = _d(eps); _, x_p = _d(ax); _, y_p = _d(ay)
    n = lib().orc_lens(pp, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       ax.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       ay.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return eps[:n], (ax + 1j * ay)[:n]


def source_centre(p: dict, t) -> np.ndarray:
    prm, pp = _d(param_vector(p))
    t, tp = _d(np.atleast_1d(t))
    wx = np.zeros_like(t); wy = np.zeros_like(t)
    lib().orc_source_centre(pp, tp, len(t), wx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            wy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return wx + 1j * wy


def poly(p: dict, w: complex, centre: complex = 0.0) -> np.ndarray:
    prm, pp = _d(param_vector(p))
    re = np.zeros(16); im = np.zeros(16)
    n = lib().orc_poly(pp, w.real, w.imag, complex(centre).real, complex(centre).imag,
                       re.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       im.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return (re + 1j * im)[: n + 1]


def roots(p: dict, w: complex, max_iter: int = 100):
    prm, pp = _d(param_vector(p))
    zr = np.zeros(16); zi = np.zeros(16)
    ok = lib().orc_roots(pp, w.real, w.imag, max_iter,
                         zr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         zi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    n = 5 if int(p.get("n_lens", 2)) == 2 else 10
    return (zr + 1j * zi)[:n], bool(ok)


def lens_map(p: dict, z) -> np.ndarray:
    prm, pp = _d(param_vector(p))
    z = np.atleast_1d(np.asarray(z, dtype=complex))
    zx, zxp = _d(z.real); zy, zyp = _d(z.imag)
    wx = np.zeros(len(z)); wy = np.zeros(len(z))
    lib().orc_lens_map(pp, zxp, zyp, len(z), wx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       wy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return wx + 1j * wy


def point_source(p: dict, grid: dict, w):
    """Returns (A, n_img, images[n, n_deg], status)."""
    prm, pp = _d(param_vector(p))
    g, gp = _d(grid_vector(grid))
    w = np.atleast_1d(np.asarray(w, dtype=complex))
    n = len(w)
    nd = 5 if int(p.get("n_lens", 2)) == 2 else 10
    wx, wxp = _d(w.real); wy, wyp = _d(w.imag)
    A = np.zeros(n); nimg = np.zeros(n, dtype=np.int32)
    zr = np.zeros(n * nd); zi = np.zeros(n * nd); st = np.zeros(n, dtype=np.uint32)
    lib().orc_point_source(pp, gp, wxp, wyp, n, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           nimg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           zr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           zi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return A, nimg, (zr + 1j * zi).reshape(n, nd), st


def sectors(p: dict, t: float, grid: dict):
    """Sectors of one epoch as an array [k, 5] = (r_lo, r_hi, th_lo, width, periodic)."""
    prm, pp = _d(param_vector(p))
    g, gp = _d(grid_vector(grid))
    out = np.zeros(64 * 5); st = np.zeros(1, dtype=np.uint32)
    n = lib().orc_sectors(pp, float(t), gp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 64,
                          st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out[: 5 * n].reshape(n, 5), int(st[0])


def magnification(params, t, grid: dict):
    """params: list of dicts (S) or one dict; t: [S, E] or [E].  Returns (A, status)."""
    if isinstance(params, dict):
        params = [params]
    prm = np.stack([param_vector(p) for p in params])
    S = prm.shape[0]
    t = np.asarray(t, dtype=np.float64).reshape(S, -1)
    E = t.shape[1]
    prm, pp = _d(prm); t, tp = _d(t)
    g, gp = _d(grid_vector(grid))
    A = np.zeros((S, E)); st = np.zeros((S, E), dtype=np.uint32)
    lib().orc_magnification(pp, S, tp, E, gp, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return A, st


def magnification_fwd(params, t, grid: dict):
    """Forward-mode derivative.  Returns (A [S,E], dA [S,E,8], status)."""
    if isinstance(params, dict):
        params = [params]
    prm = np.stack([param_vector(p) for p in params])
    S = prm.shape[0]
    t = np.asarray(t, dtype=np.float64).reshape(S, -1)
    E = t.shape[1]
    prm, pp = _d(prm); t, tp = _d(t)
    g, gp = _d(grid_vector(grid))
    A = np.zeros((S, E)); dA = np.zeros((S, E, 8)); st = np.zeros((S, E), dtype=np.uint32)
    lib().orc_magnification_fwd(pp, S, tp, E, gp, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                dA.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return A, dA, st


def limb_points(p: dict, t: float, grid: dict) -> np.ndarray:
    """Image-limb points of one epoch: [N_limb, N_deg, 3] = (r, theta, valid)."""
    prm, pp = _d(param_vector(p))
    g, gp = _d(grid_vector(grid))
    nd = 5 if int(p.get("n_lens", 2)) == 2 else 10
    out = np.zeros(int(grid["n_limb"]) * nd * 3)
    lib().orc_limb_points(pp, float(t), gp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out.reshape(int(grid["n_limb"]), nd, 3)

"""Python binding of the ICRS C ABI (include/icrs.h).

Argument marshalling only: every step of the magnification path runs in the
CUDA library ``libicrs.so``.  PyTorch supplies device memory and the current
stream.  If the library is missing the import of this module raises; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libicrs.so")

ICRS_OK, ICRS_EINVAL, ICRS_ECUDA, ICRS_ETIMEOUT, ICRS_EUNSUPPORTED = 0, 1, 2, 3, 4
ST_NONCONV, ST_IMGCOUNT, ST_SECTCAP, ST_EDGE, ST_NAN, ST_OVERFLOW, ST_LIMB, ST_ROUGH = 1, 2, 4, 8, 16, 32, 64, 128
ST_SPOT, ST_PROFILE = 1 << 16, 1 << 17

# Every symbol the header declares (checked by the CPU test suite).
EXPORTED = ("icrs_grid_default", "icrs_point_source", "icrs_magnification",
            "icrs_magnification_diag", "icrs_magnification_vjp", "icrs_chi2_grad",
            "icrs_magnification_indexed", "icrs_mlp_pack", "icrs_mlp_infer",
            "icrs_mlp_workspace_bytes", "icrs_mlp_train_step", "icrs_mlp_train_step_noalloc",
            "icrs_surrogate_features",
            "icrs_surrogate_gate_workspace_bytes", "icrs_surrogate_gate",
            "icrs_marginal_nll_workspace_bytes", "icrs_marginal_nll_grad",
            "icrs_surrogate_target", "icrs_surrogate_batch",
            "icrs_epoch_gate_workspace_bytes", "icrs_epoch_gate",
            "icrs_strerror", "icrs_abi_version")

MLP_NPARAM = 50818
MLP_PACK_BYTES = 208896
MLP_STATIC_MAX_N = 4096  # largest batch of mlp_train_step_noalloc
TARGET_SCALE = 1e4  # the network predicts 1e4 log(A / A_ps)

# Order of the 8 derivative slots of icrs_magnification_vjp / icrs_chi2_grad.
PARAM_ORDER = ("t0", "tE", "u0", "alpha", "s", "q", "rho", "u1")


class IcrsParams(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("tE", ctypes.c_double), ("u0", ctypes.c_double),
                ("alpha", ctypes.c_double), ("rho", ctypes.c_double), ("u1", ctypes.c_double),
                ("n_lens", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("s", ctypes.c_double), ("q", ctypes.c_double),
                ("q2", ctypes.c_double), ("q3", ctypes.c_double), ("s2", ctypes.c_double),
                ("s3", ctypes.c_double), ("psi", ctypes.c_double), ("u2", ctypes.c_double),
                ("a1", ctypes.c_double), ("a2", ctypes.c_double), ("a3", ctypes.c_double), ("a4", ctypes.c_double),
                ("spot_x", ctypes.c_double), ("spot_y", ctypes.c_double), ("spot_r", ctypes.c_double),
                ("spot_c", ctypes.c_double)]


class IcrsGrid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_limb", ctypes.c_int32),
                ("n_bins_r", ctypes.c_int32), ("n_bins_theta", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("uniform", ctypes.c_int32), ("n_lens", ctypes.c_int32),
                ("delta_c", ctypes.c_double), ("margin", ctypes.c_double), ("img_tol", ctypes.c_double),
                ("ld_split", ctypes.c_int32), ("grad_rule", ctypes.c_int32), ("s_fac", ctypes.c_double)]


PARAMS_DTYPE = np.dtype([("t0", "<f8"), ("tE", "<f8"), ("u0", "<f8"), ("alpha", "<f8"),
                         ("rho", "<f8"), ("u1", "<f8"), ("n_lens", "<i4"), ("reserved", "<i4"),
                         ("s", "<f8"), ("q", "<f8"), ("q2", "<f8"), ("q3", "<f8"),
                         ("s2", "<f8"), ("s3", "<f8"), ("psi", "<f8"), ("u2", "<f8"),
                         ("a1", "<f8"), ("a2", "<f8"), ("a3", "<f8"), ("a4", "<f8"),
                         ("spot_x", "<f8"), ("spot_y", "<f8"), ("spot_r", "<f8"), ("spot_c", "<f8")])
assert PARAMS_DTYPE.itemsize == ctypes.sizeof(IcrsParams)


class IcrsError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
                          f"(or python -m paper_2510_02639_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.icrs_grid_default.argtypes = [ctypes.POINTER(IcrsGrid)]
    L.icrs_grid_default.restype = None
    L.icrs_point_source.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                    vp, vp, vp, vp, vp]
    L.icrs_point_source.restype = ctypes.c_int
    L.icrs_magnification.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                     vp, vp, vp]
    L.icrs_magnification.restype = ctypes.c_int
    L.icrs_magnification_diag.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                          vp, vp, vp, vp, vp, vp]
    L.icrs_magnification_diag.restype = ctypes.c_int
    L.icrs_magnification_vjp.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                         vp, vp, vp, vp, vp, vp]
    L.icrs_magnification_vjp.restype = ctypes.c_int
    L.icrs_chi2_grad.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                 vp, vp, vp, vp, vp, vp, vp]
    L.icrs_chi2_grad.restype = ctypes.c_int
    L.icrs_marginal_nll_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    L.icrs_marginal_nll_workspace_bytes.restype = ctypes.c_size_t
    L.icrs_marginal_nll_grad.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid),
                                         vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.icrs_marginal_nll_grad.restype = ctypes.c_int
    L.icrs_magnification_indexed.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                                             ctypes.POINTER(IcrsGrid), vp, vp, vp]
    L.icrs_magnification_indexed.restype = ctypes.c_int
    L.icrs_mlp_pack.argtypes = [vp, vp, vp]
    L.icrs_mlp_pack.restype = ctypes.c_int
    L.icrs_mlp_infer.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp]
    L.icrs_mlp_infer.restype = ctypes.c_int
    L.icrs_mlp_workspace_bytes.argtypes = [ctypes.c_int]
    L.icrs_mlp_workspace_bytes.restype = ctypes.c_size_t
    L.icrs_mlp_train_step.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, vp, vp, ctypes.c_int,
                                      vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.icrs_mlp_train_step.restype = ctypes.c_int
    L.icrs_mlp_train_step_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, vp, vp, ctypes.c_int,
                                              vp, vp, vp, vp]
    L.icrs_mlp_train_step_noalloc.restype = ctypes.c_int
    L.icrs_surrogate_features.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(IcrsGrid), vp, vp, vp, vp]
    L.icrs_surrogate_features.restype = ctypes.c_int
    L.icrs_surrogate_gate_workspace_bytes.argtypes = [ctypes.c_int]
    L.icrs_surrogate_gate_workspace_bytes.restype = ctypes.c_size_t
    L.icrs_surrogate_gate.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_double, ctypes.c_float, ctypes.c_double, vp, vp, vp, vp,
                                      ctypes.c_size_t, vp]
    L.icrs_surrogate_gate.restype = ctypes.c_int
    L.icrs_surrogate_target.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp]
    L.icrs_surrogate_target.restype = ctypes.c_int
    L.icrs_surrogate_batch.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp]
    L.icrs_surrogate_batch.restype = ctypes.c_int
    L.icrs_epoch_gate_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    L.icrs_epoch_gate_workspace_bytes.restype = ctypes.c_size_t
    L.icrs_epoch_gate.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_float, ctypes.c_float, ctypes.c_double, ctypes.c_float, ctypes.c_double,
                                  vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.icrs_epoch_gate.restype = ctypes.c_int
    L.icrs_strerror.argtypes = [ctypes.c_int]
    L.icrs_strerror.restype = ctypes.c_char_p
    L.icrs_abi_version.restype = ctypes.c_int
    return L


lib = _load()


def check(rc: int):
    if rc != ICRS_OK:
        raise IcrsError(f"icrs error {rc}: {lib.icrs_strerror(rc).decode()}")


def make_grid(**kw) -> IcrsGrid:
    g = IcrsGrid()
    lib.icrs_grid_default(ctypes.byref(g))
    for k, v in kw.items():
        setattr(g, k, v)
    return g


def params_array(params) -> np.ndarray:
    """Pack a list of parameter dicts into the C struct layout."""
    a = np.zeros(len(params), dtype=PARAMS_DTYPE)
    for i, p in enumerate(params):
        for k in PARAMS_DTYPE.names:
            if k == "reserved":
                continue
            a[i][k] = p.get(k, 0)
    return a


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(x, dtype, shape=None, name="tensor"):
    """Raise ValueError unless x is a contiguous CUDA tensor of dtype (and shape)."""
    if x is None or not x.is_cuda or x.dtype != dtype or not x.is_contiguous():
        got = None if x is None else (x.dtype, x.device, x.is_contiguous())
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor, got {got}")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name}: need shape {tuple(shape)}, got {tuple(x.shape)}")
    return x


def _nsets(params_dev):
    """Number of icrs_params structs in a uint8 device tensor."""
    import torch
    _need(params_dev, torch.uint8, name="params")
    if params_dev.numel() % PARAMS_DTYPE.itemsize:
        raise ValueError("params: size is not a multiple of sizeof(icrs_params)")
    return params_dev.numel() // PARAMS_DTYPE.itemsize


def _times(t, S):
    """t: [S, E] float64 CUDA tensor; returns E."""
    import torch
    if t.dim() != 2 or t.shape[0] != S:
        raise ValueError(f"t: need shape [{S}, E], got {tuple(t.shape)}")
    _need(t, torch.float64, name="t")
    return t.shape[1]


def _stream(torch, stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def params_to_device(params, device="cuda"):
    import torch
    a = params_array(params)
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


def magnification(params_dev, t, grid: IcrsGrid, out=None, status=None, stream=None):
    """Finite-source magnification.  params_dev: uint8 device tensor holding S
    icrs_params structs; t: [S, E] float64 device tensor.  Returns (A, status)."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    if out is None:
        out = torch.empty((S, E), dtype=torch.float64, device=t.device)
    else:
        _need(out, torch.float64, (S, E), "out")
    if status is None:
        status = torch.empty((S, E), dtype=torch.int32, device=t.device)
    else:
        _need(status, torch.int32, (S, E), "status")
    check(lib.icrs_magnification(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid),
                                 _ptr(out), _ptr(status), _stream(torch, stream)))
    return out, status


def magnification_diag(params_dev, t, grid: IcrsGrid, points=False, stream=None):
    """As magnification(), plus sectors [S, E, 10, 5], counters [S, E, 16] and
    optionally the image-limb points [S, E, N_limb * N_deg, 4] per epoch."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    out = torch.empty((S, E), dtype=torch.float64, device=t.device)
    status = torch.empty((S, E), dtype=torch.int32, device=t.device)
    sect = torch.empty((S, E, 10, 5), dtype=torch.float64, device=t.device)
    cnt = torch.empty((S, E, 16), dtype=torch.int32, device=t.device)
    nd = 5 if grid.n_lens == 2 else 10
    pts = torch.empty((S, E, grid.n_limb * nd, 4), dtype=torch.float32, device=t.device) if points else None
    check(lib.icrs_magnification_diag(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid), _ptr(out),
                                      _ptr(status), _ptr(sect), _ptr(cnt), _ptr(pts), _stream(torch, stream)))
    return out, status, sect, cnt, pts


def point_source(params_dev, w, grid: IcrsGrid, n_lens=2, stream=None):
    """Point-source magnification at positions w: [S, n, 2] float64 device.
    Returns (A [S, n], images [S, n, N_deg, 2], n_img [S, n], status [S, n])."""
    import torch
    S = _nsets(params_dev)
    if w.dim() != 3 or w.shape[0] != S or w.shape[2] != 2:
        raise ValueError(f"w: need shape [{S}, n, 2], got {tuple(w.shape)}")
    _need(w, torch.float64, name="w")
    n = w.shape[1]
    nd = 5 if n_lens == 2 else 10
    A = torch.empty((S, n), dtype=torch.float64, device=w.device)
    imgs = torch.empty((S, n, nd, 2), dtype=torch.float64, device=w.device)
    nimg = torch.empty((S, n), dtype=torch.int32, device=w.device)
    st = torch.empty((S, n), dtype=torch.int32, device=w.device)
    check(lib.icrs_point_source(_ptr(params_dev), S, _ptr(w), n, ctypes.byref(grid), _ptr(A),
                                _ptr(imgs), _ptr(nimg), _ptr(st), _stream(torch, stream)))
    return A, imgs, nimg, st


def grid_from_dict(d: dict, n_lens: int = 2) -> IcrsGrid:
    return make_grid(n_r=int(d["n_r"]), n_theta=int(d["n_theta"]), n_limb=int(d["n_limb"]),
                     n_bins_r=int(d["n_bins_r"]), n_bins_theta=int(d["n_bins_theta"]),
                     max_iter=int(d["max_iter"]), uniform=int(d["uniform"]), n_lens=int(n_lens),
                     delta_c=float(d["delta_c"]), margin=float(d["margin"]),
                     img_tol=float(d["img_tol"]), ld_split=int(d.get("ld_split", 0)),
                     grad_rule=int(d.get("grad_rule", 0)), s_fac=float(d.get("s_fac", 100.0)))


def magnification_vjp(params_dev, t, grid: IcrsGrid, gA, per_epoch=False, stream=None):
    """Binary lens.  grad[s] = sum_e gA[s, e] dA[s, e]/dp over the 8 parameters
    of PARAM_ORDER.  Returns (grad [S, 8], dA [S, E, 8] or None, A [S, E],
    status [S, E])."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    _need(gA, torch.float64, (S, E), "gA")
    grad = torch.empty((S, 8), dtype=torch.float64, device=t.device)
    dA = torch.empty((S, E, 8), dtype=torch.float64, device=t.device) if per_epoch else None
    A = torch.empty((S, E), dtype=torch.float64, device=t.device)
    st = torch.empty((S, E), dtype=torch.int32, device=t.device)
    check(lib.icrs_magnification_vjp(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid), _ptr(gA),
                                     _ptr(grad), _ptr(dA), _ptr(A), _ptr(st), _stream(torch, stream)))
    return grad, dA, A, st


def chi2_grad(params_dev, t, grid: IcrsGrid, y, sigma, stream=None):
    """chi^2 = sum_e ((y - A) / sigma)^2 per set and its gradient over the 8
    parameters of PARAM_ORDER.  Returns (chi2 [S], grad [S, 8], A [S, E],
    status [S, E])."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    _need(y, torch.float64, (S, E), "y")
    _need(sigma, torch.float64, (S, E), "sigma")
    chi2 = torch.empty((S,), dtype=torch.float64, device=t.device)
    grad = torch.empty((S, 8), dtype=torch.float64, device=t.device)
    A = torch.empty((S, E), dtype=torch.float64, device=t.device)
    st = torch.empty((S, E), dtype=torch.int32, device=t.device)
    check(lib.icrs_chi2_grad(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid), _ptr(y), _ptr(sigma),
                             _ptr(chi2), _ptr(grad), _ptr(A), _ptr(st), _stream(torch, stream)))
    return chi2, grad, A, st


def marginal_nll_grad(params_dev, t, grid: IcrsGrid, F, sigma, prior, grad=True, workspace=None, stream=None):
    """Linear-flux marginalised NLL per light curve (icrs_marginal_nll_grad).
    F, sigma: [S, E] float64; prior: [S, 4] float64 (mu_S, mu_base,
    lambda_S, lambda_base).  Returns (nll [S], grad [S, 8] or None,
    fluxes [S, 2], A [S, E], status [S, E])."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    _need(F, torch.float64, (S, E), "F")
    _need(sigma, torch.float64, (S, E), "sigma")
    _need(prior, torch.float64, (S, 4), "prior")
    nll = torch.empty((S,), dtype=torch.float64, device=t.device)
    g = torch.empty((S, 8), dtype=torch.float64, device=t.device) if grad else None
    fl = torch.empty((S, 2), dtype=torch.float64, device=t.device)
    A = torch.empty((S, E), dtype=torch.float64, device=t.device)
    st = torch.empty((S, E), dtype=torch.int32, device=t.device)
    nb = int(lib.icrs_marginal_nll_workspace_bytes(S, E))
    if workspace is None or workspace.numel() < nb:
        workspace = torch.empty(max(nb, 8), dtype=torch.uint8, device=t.device)
    check(lib.icrs_marginal_nll_grad(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid), _ptr(F), _ptr(sigma),
                                     _ptr(prior), _ptr(nll), _ptr(g), _ptr(fl), _ptr(A), _ptr(st), _ptr(workspace),
                                     nb, _stream(torch, stream)))
    return nll, g, fl, A, st


def pack_binary(theta):
    """Device-side packing of binary-lens parameters theta [S, 8] (PARAM_ORDER,
    float64) into icrs_params structs (uint8 tensor)."""
    import torch
    S = theta.shape[0]
    buf = torch.zeros((S, PARAMS_DTYPE.itemsize // 8), dtype=torch.float64, device=theta.device)
    th = theta.detach()
    # struct order: t0, tE, u0, alpha, rho, u1, (n_lens, reserved), s, q, ...
    for dst, src in ((0, 0), (1, 1), (2, 2), (3, 3), (4, 6), (5, 7), (7, 4), (8, 5)):
        buf[:, dst] = th[:, src]
    buf.view(torch.int32)[:, 12] = 2
    return buf.view(torch.uint8).reshape(-1)


def _autograd_function():
    import torch

    class Magnification(torch.autograd.Function):
        """A [S, E] = ICRS magnification of binary-lens parameters theta [S, 8]
        (PARAM_ORDER) at epochs t [S, E].  Backward: icrs_magnification_vjp,
        which recomputes the rays of every epoch."""

        @staticmethod
        def forward(ctx, theta, t, grid):
            pd = pack_binary(theta)
            A, st = magnification(pd, t, grid)
            ctx.save_for_backward(t)
            ctx.pd = pd
            ctx.grid = grid
            ctx.status = st
            return A

        @staticmethod
        def backward(ctx, gA):
            (t,) = ctx.saved_tensors
            grad, _, _, _ = magnification_vjp(ctx.pd, t, ctx.grid, gA.contiguous().to(torch.float64))
            return grad, None, None

    return Magnification


_MAG_FN = None


def magnification_ad(theta, t, grid: IcrsGrid):
    """Differentiable magnification (torch.autograd): theta [S, 8] float64 on
    the device in PARAM_ORDER, t [S, E] float64.  Binary lens."""
    global _MAG_FN
    if _MAG_FN is None:
        _MAG_FN = _autograd_function()
    return _MAG_FN.apply(theta, t, grid)


def magnification_indexed(params_dev, t, grid: IcrsGrid, items, n, A, status=None, stream=None):
    """ICRS on items[0:n] (indices s * E + e) of the [S, E] problem; writes
    A[s, e] (and status) for those items only."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    _need(items, torch.int32, name="items")
    if not 0 <= int(n) <= items.numel():
        raise ValueError("items: n out of range")
    _need(A, torch.float64, name="A")
    if A.numel() != S * E:
        raise ValueError("A: need S * E values")
    if status is not None:
        _need(status, torch.int32, name="status")
        if status.numel() != S * E:
            raise ValueError("status: need S * E values")
    check(lib.icrs_magnification_indexed(_ptr(params_dev), S, _ptr(t), E, _ptr(items), int(n), ctypes.byref(grid),
                                         _ptr(A), _ptr(status), _stream(torch, stream)))
    return A


def mlp_pack(theta, pack=None, stream=None):
    import torch
    if pack is None:
        pack = torch.empty(MLP_PACK_BYTES, dtype=torch.uint8, device=theta.device)
    check(lib.icrs_mlp_pack(_ptr(theta), _ptr(pack), _stream(torch, stream)))
    return pack


def mlp_infer(pack, theta, feat, out=None, err=None, stream=None):
    """feat [n, 8] float32 -> (mu, s) [n, 2] float32."""
    import torch
    n = feat.shape[0]
    _need(feat, torch.float32, (n, 8), "feat")
    if out is None:
        out = torch.empty((n, 2), dtype=torch.float32, device=feat.device)
    check(lib.icrs_mlp_infer(_ptr(pack), _ptr(theta), _ptr(feat), n, _ptr(out), _ptr(err), _stream(torch, stream)))
    return out


def mlp_workspace(n, device="cuda"):
    import torch
    nb = int(lib.icrs_mlp_workspace_bytes(int(n)))
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


def mlp_train_step(theta, m, v, pack, step, lr, feat, target, workspace=None, grad=None, loss=None, err=None,
                   stream=None):
    """One training step (Adam if lr > 0).  Returns (grad, loss) tensors
    (grad/loss may be None when not requested)."""
    import torch
    n = feat.shape[0]
    _need(feat, torch.float32, (n, 8), "feat")
    _need(target, torch.float32, name="target")
    if target.numel() != n:
        raise ValueError("target: need one value per feature row")
    if workspace is None:
        workspace = mlp_workspace(n, feat.device)
    check(lib.icrs_mlp_train_step(_ptr(theta), _ptr(m), _ptr(v), _ptr(pack), int(step), float(lr), _ptr(feat),
                                  _ptr(target), n, _ptr(grad), _ptr(loss), _ptr(workspace), workspace.numel(),
                                  _ptr(err), _stream(torch, stream)))
    return grad, loss


def surrogate_features(params_dev, t, grid: IcrsGrid, stream=None):
    """Returns (features [S*E, 8] f32, A_ps [S*E] f64, status [S*E] int32)."""
    import torch
    S = _nsets(params_dev)
    E = _times(t, S)
    feat = torch.empty((S * E, 8), dtype=torch.float32, device=t.device)
    Aps = torch.empty((S * E,), dtype=torch.float64, device=t.device)
    st = torch.empty((S * E,), dtype=torch.int32, device=t.device)
    check(lib.icrs_surrogate_features(_ptr(params_dev), S, _ptr(t), E, ctypes.byref(grid), _ptr(feat), _ptr(Aps),
                                      _ptr(st), _stream(torch, stream)))
    return feat, Aps, st


def surrogate_gate(pred, feat, A_ps, st_ps, sigma_max, mu_max, b_max, caustic_min, A_max=1e300, rho_min=0.0,
                   A_small=1e300, A=None, stream=None):
    """Returns (A [n] f64 with accepted epochs filled, routed_idx [n] int32,
    n_routed [1] int32 device)."""
    import torch
    n = pred.shape[0]
    dev = pred.device
    if A is None:
        A = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    idx = torch.empty((n,), dtype=torch.int32, device=dev)
    nr = torch.zeros((1,), dtype=torch.int32, device=dev)
    ws = torch.empty(max(int(lib.icrs_surrogate_gate_workspace_bytes(n)), 256), dtype=torch.uint8, device=dev)
    check(lib.icrs_surrogate_gate(_ptr(pred), _ptr(feat), _ptr(A_ps), _ptr(st_ps), n, float(sigma_max),
                                  float(mu_max), float(b_max), float(caustic_min), float(A_max), float(rho_min),
                                  float(A_small), _ptr(A), _ptr(idx),
                                  _ptr(nr), _ptr(ws),
                                  ws.numel(), _stream(torch, stream)))
    return A, idx, nr


def mlp_train_step_noalloc(theta, m, v, pack, step, lr, feat, target, grad=None, loss=None, err=None, stream=None):
    """As mlp_train_step, with the library's static scratch (n <= 4096);
    overlapping calls on one device race on that scratch."""
    import torch
    n = feat.shape[0]
    _need(feat, torch.float32, (n, 8), "feat")
    _need(target, torch.float32, name="target")
    if target.numel() != n:
        raise ValueError("target: need one value per feature row")
    check(lib.icrs_mlp_train_step_noalloc(_ptr(theta), _ptr(m), _ptr(v), _ptr(pack), int(step), float(lr),
                                          _ptr(feat), _ptr(target), n, _ptr(grad), _ptr(loss), _ptr(err),
                                          _stream(torch, stream)))
    return grad, loss


def epoch_gate(feat, A_ps, st_ps, S, E, n_ext, mode, b_max, caustic_min, A_max=1e300, rho_min=0.0, A_small=1e300,
               A=None, stream=None):
    """Non-learned epoch preselection (icrs_epoch_gate).  feat [S*E, 8],
    A_ps [S*E], st_ps [S*E] from surrogate_features.  Returns (A [S*E] with
    the non-routed epochs filled, routed_idx [S*E] int32, n_routed [1])."""
    import torch
    n = S * E
    dev = feat.device
    if A is None:
        A = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    idx = torch.empty((max(n, 1),), dtype=torch.int32, device=dev)
    nr = torch.zeros((1,), dtype=torch.int32, device=dev)
    ws = torch.empty(max(int(lib.icrs_epoch_gate_workspace_bytes(S, E)), 256), dtype=torch.uint8, device=dev)
    check(lib.icrs_epoch_gate(_ptr(feat), _ptr(A_ps), _ptr(st_ps), int(S), int(E), int(n_ext), int(mode),
                              float(b_max), float(caustic_min), float(A_max), float(rho_min), float(A_small),
                              _ptr(A), _ptr(idx), _ptr(nr), _ptr(ws), ws.numel(), _stream(torch, stream)))
    return A, idx, nr


def surrogate_target(A, A_ps, feat, out=None, stream=None):
    """target [n] float32 = 1e4 log(A / A_ps) - feat[:, 7] (icrs_surrogate_target)."""
    import torch
    n = A.numel()
    _need(A, torch.float64, name="A")
    _need(A_ps, torch.float64, (n,), "A_ps")
    _need(feat, torch.float32, (n, 8), "feat")
    if out is None:
        out = torch.empty((n,), dtype=torch.float32, device=A.device)
    check(lib.icrs_surrogate_target(_ptr(A), _ptr(A_ps), _ptr(feat), n, _ptr(out), _stream(torch, stream)))
    return out


def surrogate_batch(feat, target, idx, out_feat=None, out_target=None, stream=None):
    """Rows idx of (feat [N, 8], target [N]) into (out_feat [n, 8], out_target [n])."""
    import torch
    n = idx.numel()
    _need(idx, torch.int32, name="idx")
    _need(feat, torch.float32, name="feat")
    _need(target, torch.float32, name="target")
    if feat.dim() != 2 or feat.shape[1] != 8 or target.numel() != feat.shape[0]:
        raise ValueError("feat / target: need [N, 8] and [N]")
    if out_feat is None:
        out_feat = torch.empty((n, 8), dtype=torch.float32, device=feat.device)
    if out_target is None:
        out_target = torch.empty((n,), dtype=torch.float32, device=feat.device)
    check(lib.icrs_surrogate_batch(_ptr(feat), _ptr(target), _ptr(idx), n, _ptr(out_feat), _ptr(out_target),
                                   _stream(torch, stream)))
    return out_feat, out_target

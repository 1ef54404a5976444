"""Thin Python binding of the C ABI in include/ddm.h.

Argument marshalling only: every step of the computation runs in the CUDA
library (libddm_gb300.so, built for sm_103a).  Device buffers are torch CUDA
tensors (float64, contiguous); the library is loaded from the package's
_build directory and there is no fallback: a missing library raises.

The functions carry the C names (ddm_create, ddm_build_tree, ddm_matvec,
ddm_history_apply, ddm_rhs, ddm_gmres_solve, ddm_sif, ...); ``Context`` and
``Tree`` wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

DDM_OK, DDM_EINVAL, DDM_ENOMEM, DDM_ENOTCONV, DDM_ETIMEOUT, DDM_ECUDA, DDM_PENDING, DDM_ECANCELED = range(8)
MODE_FMM, MODE_DENSE, MODE_PRECISE = 0, 1, 16
SYS_PRESSURE, SYS_IMPERMEABLE, SYS_RATE = 0, 1, 2
_MODES = {"fmm": MODE_FMM, "dense": MODE_DENSE, "fmm+precise": MODE_FMM | MODE_PRECISE,
          "dense+precise": MODE_DENSE | MODE_PRECISE}
_SYSTEMS = {"pressure": SYS_PRESSURE, "impermeable": SYS_IMPERMEABLE, "rate": SYS_RATE}
EXPORTS = ("ddm_create", "ddm_destroy", "ddm_last_error", "ddm_device_check", "ddm_build_tree", "ddm_tree_destroy",
           "ddm_tree_get_info", "ddm_matvec", "ddm_history_apply", "ddm_rhs", "ddm_gmres_solve", "ddm_sif",
           "ddm_profile", "ddm_profile_read", "ddm_batch_create", "ddm_batch_destroy", "ddm_batch_matvec",
           "ddm_batch_gmres_solve", "ddm_server_create", "ddm_submit", "ddm_poll", "ddm_server_destroy",
           "ddm_matvec_dense_static", "ddm_set_wait_limit", "ddm_build_tree_params", "ddm_autotune",
           "ddm_set_m2l_compression", "ddm_set_history_compression", "ddm_server_cancel",
           "ddm_server_get_stats", "ddm_grow", "ddm_server_set_mode")
STATIC_MAX_ELEMENTS = 65536
NSTAGES = 10
STAGES = ("prep", "self_blocks", "up", "m2l_ops", "m2l", "down", "leaf", "dense", "krylov", "tree")


class ddm_material(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("G", "nu", "nu_u", "B", "perm", "visc")]


class ddm_fmm_params(ctypes.Structure):
    _fields_ = [("n_cheb", ctypes.c_int), ("leaf_size", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("quad_near", ctypes.c_int), ("adaptive", ctypes.c_int)]


class ddm_tree_info(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int64), ("depth", ctypes.c_int), ("n_cells", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_m2l_pairs", ctypes.c_int64), ("n_p2p_pairs", ctypes.c_int64),
                ("root_half_width", ctypes.c_double), ("leaf_level_min", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("max_leaf_records", ctypes.c_int)]


class ddm_loads(ctypes.Structure):
    _fields_ = [("sigma_H", ctypes.c_double), ("sigma_h", ctypes.c_double), ("p_f", ctypes.c_double),
                ("p0", ctypes.c_double), ("system", ctypes.c_int)]


class ddm_gmres_params(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("mode", ctypes.c_int)]


class ddm_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d_xy", ctypes.c_void_p), ("loads", ddm_loads), ("dt", ctypes.c_double),
                ("steps", ctypes.c_int), ("d_x", ctypes.c_void_p)]


class ddm_server_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("solves", ctypes.c_int64), ("ms_admit", ctypes.c_double),
                ("ms_history", ctypes.c_double), ("ms_setup", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("ms_other", ctypes.c_double)]


class ddm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("steps_done", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ddm_gmres_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libddm_gb300.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            _build.build()
        L = ctypes.CDLL(path)
        L.ddm_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(ddm_material), ctypes.POINTER(ddm_fmm_params), _VP]
        L.ddm_destroy.argtypes = [_VP]
        L.ddm_destroy.restype = None
        L.ddm_last_error.argtypes = [_VP]
        L.ddm_last_error.restype = ctypes.c_char_p
        L.ddm_build_tree.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.POINTER(_VP)]
        L.ddm_tree_destroy.argtypes = [_VP]
        L.ddm_tree_destroy.restype = None
        L.ddm_tree_get_info.argtypes = [_VP, ctypes.POINTER(ddm_tree_info)]
        L.ddm_matvec.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP, ctypes.c_int]
        L.ddm_history_apply.argtypes = [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int, _VP, ctypes.c_int]
        L.ddm_rhs.argtypes = [_VP, _VP, ctypes.POINTER(ddm_loads), _VP, _VP]
        L.ddm_gmres_solve.argtypes = [_VP, _VP, ctypes.c_double, _VP, _VP, ctypes.POINTER(ddm_gmres_params),
                                      ctypes.POINTER(ddm_gmres_info)]
        L.ddm_sif.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP]
        L.ddm_profile.argtypes = [_VP, ctypes.c_int]
        L.ddm_set_wait_limit.argtypes = [_VP, ctypes.c_int64]
        L.ddm_set_m2l_compression.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
        L.ddm_set_history_compression.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.ddm_build_tree_params.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.POINTER(ddm_fmm_params), ctypes.POINTER(_VP)]
        L.ddm_autotune.argtypes = [_VP, _VP, ctypes.c_int64, _VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(ddm_fmm_params), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
        L.ddm_matvec_dense_static.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _VP, _VP]
        L.ddm_server_create.argtypes = [_VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_VP)]
        L.ddm_submit.argtypes = [_VP, ctypes.POINTER(ddm_request), ctypes.POINTER(ctypes.c_uint64)]
        L.ddm_poll.argtypes = [_VP, ctypes.c_uint64, ctypes.POINTER(ddm_result)]
        L.ddm_server_destroy.argtypes = [_VP]
        L.ddm_server_destroy.restype = None
        L.ddm_server_cancel.argtypes = [_VP]
        L.ddm_server_set_mode.argtypes = [_VP, ctypes.c_int]
        L.ddm_grow.argtypes = [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP,
                               ctypes.POINTER(ctypes.c_int64), _VP, _VP]
        L.ddm_server_get_stats.argtypes = [_VP, ctypes.POINTER(ddm_server_stats)]
        L.ddm_batch_create.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)]
        L.ddm_batch_destroy.argtypes = [_VP]
        L.ddm_batch_destroy.restype = None
        L.ddm_batch_matvec.argtypes = [_VP, _VP, ctypes.c_double, _VP, _VP, ctypes.c_int]
        L.ddm_batch_gmres_solve.argtypes = [_VP, _VP, ctypes.c_double, _VP, _VP, ctypes.POINTER(ddm_gmres_params),
                                            ctypes.POINTER(ddm_gmres_info)]
        L.ddm_profile_read.argtypes = [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        for name in EXPORTS:      # every entry point returns ddm_status unless set above
            fn = getattr(L, name)
            if name not in ("ddm_destroy", "ddm_tree_destroy", "ddm_batch_destroy", "ddm_server_destroy",
                            "ddm_last_error"):
                fn.restype = ctypes.c_int
        _lib = L
        return L


class DDMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ddm status {status}: {msg}")
        self.status = status


def _check(ctx_ptr, st, what):
    if st != DDM_OK:
        msg = load().ddm_last_error(ctx_ptr).decode(errors="replace") if ctx_ptr else ""
        raise DDMError(st, f"{what}: {msg}")


def _dev(t: torch.Tensor, n=None, name="tensor") -> int:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return t.data_ptr()


# ---------------------------------------------------------------- C names
def _tree_kind(adaptive):
    """ddm_fmm_params.adaptive: False / 0 uniform, True / 1 adaptive, "auto" / 2
    both built and the one the library's cost model prefers kept."""
    if adaptive == "auto":
        return 2
    if adaptive in (0, 1, 2):
        return int(adaptive)
    raise ValueError(f"adaptive must be False, True or 'auto', not {adaptive!r}")


def ddm_create(material, n_cheb=8, leaf_size=32, max_depth=0, quad_near=6, stream=None, adaptive=False):
    L = load()
    if isinstance(material, dict):
        material = [material[k] for k in ("G", "nu", "nu_u", "B", "perm", "visc")]
    m = ddm_material(*[float(v) for v in material])
    p = ddm_fmm_params(int(n_cheb), int(leaf_size), int(max_depth), int(quad_near), _tree_kind(adaptive))
    s = (stream or torch.cuda.current_stream()).cuda_stream
    out = _VP()
    st = L.ddm_create(ctypes.byref(out), ctypes.byref(m), ctypes.byref(p), _VP(s))
    if st != DDM_OK:
        raise DDMError(st, "ddm_create failed (invalid material or parameters?)")
    return out


def ddm_destroy(ctx):
    load().ddm_destroy(ctx)


def ddm_build_tree(ctx, xy: torch.Tensor):
    n = xy.numel() // 4
    out = _VP()
    _check(ctx, load().ddm_build_tree(ctx, _VP(_dev(xy, 4 * n, "xy")), n, ctypes.byref(out)), "ddm_build_tree")
    return out


def ddm_build_tree_params(ctx, xy: torch.Tensor, n_cheb=0, leaf_size=0, max_depth=0, quad_near=0, adaptive=False):
    """Tree with its own FMM parameters (order, leaf size, quad_near: 0 = the
    context's; max_depth and adaptive as given)."""
    n = xy.numel() // 4
    out = _VP()
    prm = ddm_fmm_params(int(n_cheb), int(leaf_size), int(max_depth), int(quad_near), _tree_kind(adaptive))
    _check(ctx, load().ddm_build_tree_params(ctx, _VP(_dev(xy, 4 * n, "xy")), n, ctypes.byref(prm), ctypes.byref(out)),
           "ddm_build_tree_params")
    return out


def ddm_autotune(ctx, xy: torch.Tensor, x: torch.Tensor, dt, orders=None, leaves=None, max_rel_err=1e-3) -> dict:
    """Fastest (order, leaf size, tree kind) for this problem within the error bound."""
    n = xy.numel() // 4
    o = (ctypes.c_int * len(orders))(*orders) if orders else None
    lv = (ctypes.c_int * len(leaves))(*leaves) if leaves else None
    best = ddm_fmm_params()
    ms, err = ctypes.c_double(), ctypes.c_double()
    _check(ctx, load().ddm_autotune(ctx, _VP(_dev(xy, 4 * n, "xy")), n, _VP(_dev(x, 3 * n, "x")), float(dt), o,
                                    len(orders) if orders else 0, lv, len(leaves) if leaves else 0,
                                    float(max_rel_err), ctypes.byref(best), ctypes.byref(ms), ctypes.byref(err)),
           "ddm_autotune")
    return {"n_cheb": best.n_cheb, "leaf_size": best.leaf_size, "adaptive": bool(best.adaptive), "ms": ms.value,
            "err": err.value}


def ddm_tree_destroy(tree):
    load().ddm_tree_destroy(tree)


def ddm_tree_get_info(tree) -> dict:
    info = ddm_tree_info()
    st = load().ddm_tree_get_info(tree, ctypes.byref(info))
    if st != DDM_OK:
        raise DDMError(st, "ddm_tree_get_info")
    return {k: getattr(info, k) for k, _ in ddm_tree_info._fields_}


def ddm_matvec(ctx, tree, tau_lo, tau_hi, x, y, mode=MODE_FMM):
    n = y.numel()
    _check(ctx, load().ddm_matvec(ctx, tree, float(tau_lo), float(tau_hi), _VP(_dev(x, n, "x")),
                                  _VP(_dev(y, n, "y")), int(mode)), "ddm_matvec")


def ddm_history_apply(ctx, tree, hist, times, H, rhs, mode=MODE_FMM):
    tt = (ctypes.c_double * (H + 2))(*[float(v) for v in times])
    hp = _VP(_dev(hist, None, "hist")) if H > 0 else _VP(0)
    _check(ctx, load().ddm_history_apply(ctx, tree, hp, tt, int(H), _VP(_dev(rhs, None, "rhs")), int(mode)),
           "ddm_history_apply")


def ddm_rhs(ctx, tree, sigma_H, sigma_h, p_f, p0, system, rhs, pf=None):
    ld = ddm_loads(float(sigma_H), float(sigma_h), float(p_f), float(p0), int(system))
    pp = _VP(_dev(pf, None, "pf")) if pf is not None else _VP(0)
    _check(ctx, load().ddm_rhs(ctx, tree, ctypes.byref(ld), pp, _VP(_dev(rhs, None, "rhs"))), "ddm_rhs")


def ddm_gmres_solve(ctx, tree, dt, rhs, x, system=SYS_PRESSURE, restart=50, max_iters=1000, tol=1e-6,
                    mode=MODE_FMM, raise_on_notconv=True) -> dict:
    prm = ddm_gmres_params(int(system), int(restart), int(max_iters), float(tol), int(mode))
    info = ddm_gmres_info()
    st = load().ddm_gmres_solve(ctx, tree, float(dt), _VP(_dev(rhs, None, "rhs")), _VP(_dev(x, None, "x")),
                                ctypes.byref(prm), ctypes.byref(info))
    res = {k: getattr(info, k) for k, _ in ddm_gmres_info._fields_}
    if st == DDM_ENOTCONV and not raise_on_notconv:
        return res
    _check(ctx, st, "ddm_gmres_solve")
    return res


def ddm_sif(ctx, tree, x, tips: torch.Tensor, KI, KII):
    n = tips.numel()
    if not (tips.is_cuda and tips.dtype == torch.int64 and tips.is_contiguous()):
        raise ValueError("tips must be a contiguous int64 CUDA tensor")
    _check(ctx, load().ddm_sif(ctx, tree, _VP(_dev(x, None, "x")), _VP(tips.data_ptr()), int(n),
                               _VP(_dev(KI, n, "KI")), _VP(_dev(KII, n, "KII"))), "ddm_sif")


def ddm_profile(ctx, enable=True):
    _check(ctx, load().ddm_profile(ctx, int(bool(enable))), "ddm_profile")


def ddm_device_check(ctx):
    """Synchronise the context stream; raise DDMError (DDM_ETIMEOUT) if a
    bounded device wait expired since the last check."""
    _check(ctx, load().ddm_device_check(ctx), "ddm_device_check")


def ddm_set_wait_limit(ctx, polls=0):
    """Poll limit of the GMRES grid barriers (0 = the default)."""
    _check(ctx, load().ddm_set_wait_limit(ctx, int(polls)), "ddm_set_wait_limit")


def ddm_set_m2l_compression(ctx, mode=2, rank=0):
    """Compressed M2L operators: mode 0 never, 1 always (n >= 8), 2 automatic;
    rank 0 = the default per order."""
    _check(ctx, load().ddm_set_m2l_compression(ctx, int(mode), int(rank)), "ddm_set_m2l_compression")


def ddm_set_history_compression(ctx, exact_steps=0, nodes=10, ratio=2.0):
    """Time-compressed history sum: exact_steps most recent steps exact (0 =
    off), older steps interpolated in log time at `nodes` points per block."""
    _check(ctx, load().ddm_set_history_compression(ctx, int(exact_steps), int(nodes), float(ratio)),
           "ddm_set_history_compression")


def ddm_grow(ctx, xy: torch.Tensor, x: torch.Tensor, tips: torch.Tensor, ends: torch.Tensor, K_Ic):
    """One growth step: returns (grown geometry 4 x n_out, theta, K_eq);
    tips (int64) and ends (int32) are updated in place."""
    n = xy.numel() // 4
    m = tips.numel()
    assert tips.dtype == torch.int64 and ends.dtype == torch.int32 and tips.is_contiguous() and ends.is_contiguous()
    out = torch.empty(4 * (n + m), dtype=torch.float64, device="cuda")
    theta = torch.empty(max(m, 1), dtype=torch.float64, device="cuda")
    keq = torch.empty_like(theta)
    n_out = ctypes.c_int64(0)
    _check(ctx, load().ddm_grow(ctx, _VP(_dev(xy, 4 * n, "xy")), n, _VP(_dev(x, 3 * n, "x")), _VP(tips.data_ptr()),
                                _VP(ends.data_ptr()), m, float(K_Ic), _VP(out.data_ptr()), ctypes.byref(n_out),
                                _VP(theta.data_ptr()), _VP(keq.data_ptr())), "ddm_grow")
    n2 = n_out.value
    return out[:4 * n2].view(4, n2), theta[:m], keq[:m]


def ddm_profile_read(ctx) -> dict:
    ms = (ctypes.c_double * NSTAGES)()
    n = (ctypes.c_int64 * NSTAGES)()
    _check(ctx, load().ddm_profile_read(ctx, ms, n), "ddm_profile_read")
    return {STAGES[k]: (ms[k], n[k]) for k in range(NSTAGES)}


def ddm_matvec_dense_static(ctx, xy, tau_lo, tau_hi, x, y):
    """Allocation-free dense product (see include/ddm.h): y = [K(hi) - K(lo)] x
    for the elements xy (4N), using the library's fixed scratch array."""
    n = xy.numel() // 4
    _check(ctx, load().ddm_matvec_dense_static(ctx, _VP(_dev(xy, 4 * n, "xy")), n, float(tau_lo), float(tau_hi),
                                               _VP(_dev(x, 3 * n, "x")), _VP(_dev(y, 3 * n, "y"))),
           "ddm_matvec_dense_static")


def ddm_batch_create(ctx, trees):
    arr = (_VP * len(trees))(*[t for t in trees])
    out = _VP()
    _check(ctx, load().ddm_batch_create(ctx, arr, len(trees), ctypes.byref(out)), "ddm_batch_create")
    return out


def ddm_batch_destroy(batch):
    load().ddm_batch_destroy(batch)


def ddm_batch_matvec(ctx, batch, dt, x, y, mode=MODE_FMM):
    _check(ctx, load().ddm_batch_matvec(ctx, batch, float(dt), _VP(_dev(x, None, "x")), _VP(_dev(y, None, "y")),
                                        int(mode)), "ddm_batch_matvec")


def ddm_batch_gmres_solve(ctx, batch, n, dt, rhs, x, system=SYS_PRESSURE, restart=50, max_iters=1000, tol=1e-6,
                          mode=MODE_FMM, raise_on_notconv=True):
    prm = ddm_gmres_params(int(system), int(restart), int(max_iters), float(tol), int(mode))
    infos = (ddm_gmres_info * n)()
    st = load().ddm_batch_gmres_solve(ctx, batch, float(dt), _VP(_dev(rhs, None, "rhs")), _VP(_dev(x, None, "x")),
                                      ctypes.byref(prm), infos)
    res = [{k: getattr(i, k) for k, _ in ddm_gmres_info._fields_} for i in infos]
    if st == DDM_ENOTCONV and not raise_on_notconv:
        return res
    _check(ctx, st, "ddm_batch_gmres_solve")
    return res


def ddm_server_create(ctx, budget_bytes=0, max_active=64, tol=1e-5):
    out = _VP()
    _check(ctx, load().ddm_server_create(ctx, int(budget_bytes), int(max_active), float(tol), ctypes.byref(out)),
           "ddm_server_create")
    return out


def ddm_submit(server, xy: torch.Tensor, x_out: torch.Tensor, dt, steps, sigma_H=0.0, sigma_h=0.0, p_f=0.0, p0=0.0,
               system=SYS_PRESSURE) -> int:
    n = xy.numel() // 4
    req = ddm_request(n, _dev(xy, 4 * n, "xy"), ddm_loads(float(sigma_H), float(sigma_h), float(p_f), float(p0),
                                                          int(system)), float(dt), int(steps), _dev(x_out, 3 * n, "x"))
    t = ctypes.c_uint64()
    st = load().ddm_submit(server, ctypes.byref(req), ctypes.byref(t))
    if st != DDM_OK:
        raise DDMError(st, "ddm_submit")
    return t.value


def ddm_poll(server, ticket) -> dict:
    r = ddm_result()
    st = load().ddm_poll(server, int(ticket), ctypes.byref(r))
    d = {k: getattr(r, k) for k, _ in ddm_result._fields_}
    d["poll"] = st
    return d


def ddm_server_cancel(server):
    st = load().ddm_server_cancel(server)
    if st:
        raise DDMError(st, "ddm_server_cancel failed")


def ddm_server_destroy(server):
    load().ddm_server_destroy(server)


class Server:
    """Continuous-batching request loop (see include/ddm.h)."""

    def __init__(self, ctx: "Context", budget_bytes=0, max_active=64, tol=1e-5):
        self.ptr = ddm_server_create(ctx.ptr, budget_bytes, max_active, tol)
        self._keep = {}

    def submit(self, xy, x_out, dt, steps, system="pressure", **loads) -> int:
        t = ddm_submit(self.ptr, xy, x_out, dt, steps, system=_SYSTEMS[system], **loads)
        self._keep[t] = (xy, x_out)
        return t

    def poll(self, ticket) -> dict:
        return ddm_poll(self.ptr, ticket)

    def stats(self) -> dict:
        s = ddm_server_stats()
        st = load().ddm_server_get_stats(self.ptr, ctypes.byref(s))
        if st:
            raise DDMError(st, "ddm_server_get_stats failed")
        return {k: getattr(s, k) for k, _ in ddm_server_stats._fields_}

    def set_mode(self, mode="fmm"):
        """Product mode of later rounds: "fmm" or "dense"."""
        st = load().ddm_server_set_mode(self.ptr, _MODES[mode])
        if st:
            raise DDMError(st, "ddm_server_set_mode: fmm or dense")

    def cancel(self):
        """Cancel every unfinished request (status DDM_ECANCELED)."""
        ddm_server_cancel(self.ptr)

    def close(self):
        if self.ptr:
            ddm_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- wrappers
class Tree:
    def __init__(self, ctx: "Context", xy: torch.Tensor, n_cheb=0, leaf_size=0, adaptive=None, max_depth=None):
        self.ctx = ctx
        self.n = xy.numel() // 4
        if n_cheb or leaf_size or adaptive is not None or max_depth is not None:
            self.ptr = ddm_build_tree_params(ctx.ptr, xy, n_cheb, leaf_size,
                                             ctx.max_depth if max_depth is None else max_depth, 0,
                                             ctx.adaptive if adaptive is None else adaptive)
        else:
            self.ptr = ddm_build_tree(ctx.ptr, xy)

    def info(self) -> dict:
        return ddm_tree_get_info(self.ptr)

    def close(self):
        if self.ptr:
            ddm_tree_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent problems solved together (one graph launch per product)."""

    def __init__(self, ctx: "Context", trees):
        self.ctx = ctx
        self.trees = list(trees)
        self.sizes = [t.n for t in self.trees]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + 3 * n)
        self.ptr = ddm_batch_create(ctx.ptr, [t.ptr for t in self.trees])

    def matvec(self, x, dt, mode="fmm", out=None):
        out = torch.empty_like(x) if out is None else out
        ddm_batch_matvec(self.ctx.ptr, self.ptr, dt, x, out, _MODES[mode])
        return out

    def gmres_solve(self, dt, rhs, x=None, system="pressure", restart=50, max_iters=1000, tol=1e-6, mode="fmm",
                    raise_on_notconv=True):
        x = torch.zeros(self.offsets[-1], dtype=torch.float64, device="cuda") if x is None else x
        infos = ddm_batch_gmres_solve(self.ctx.ptr, self.ptr, len(self.trees), dt, rhs, x, _SYSTEMS[system], restart,
                                      max_iters, tol, _MODES[mode], raise_on_notconv)
        return x, infos

    def close(self):
        if self.ptr:
            ddm_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library context on the current CUDA device and stream."""

    def __init__(self, material, n_cheb=8, leaf_size=32, max_depth=0, quad_near=6, stream=None, adaptive=False):
        self.adaptive, self.max_depth = adaptive, int(max_depth)
        self.ptr = ddm_create(material, n_cheb, leaf_size, max_depth, quad_near, stream, adaptive)

    def build_tree(self, xy: torch.Tensor, n_cheb=0, leaf_size=0, adaptive=None, max_depth=None) -> Tree:
        """Quadtree of the elements (adaptive / max_depth: None = the context's)."""
        return Tree(self, xy.contiguous(), n_cheb, leaf_size, adaptive, max_depth)

    def autotune(self, xy: torch.Tensor, x: torch.Tensor, dt, orders=None, leaves=None, max_rel_err=1e-3) -> dict:
        return ddm_autotune(self.ptr, xy.contiguous(), x, dt, orders, leaves, max_rel_err)

    def matvec(self, tree: Tree, x, tau_lo=0.0, tau_hi=1.0, mode="fmm", out=None):
        out = torch.empty_like(x) if out is None else out
        ddm_matvec(self.ptr, tree.ptr, tau_lo, tau_hi, x, out, _MODES[mode])
        return out

    def history_apply(self, tree: Tree, hist, times, rhs, mode="fmm"):
        H = 0 if hist is None else hist.shape[0]
        ddm_history_apply(self.ptr, tree.ptr, hist, times, H, rhs, _MODES[mode])
        return rhs

    def rhs(self, tree: Tree, sigma_H=0.0, sigma_h=0.0, p_f=0.0, p0=0.0, system="pressure", pf=None, out=None):
        out = torch.empty(3 * tree.n, dtype=torch.float64, device="cuda") if out is None else out
        ddm_rhs(self.ptr, tree.ptr, sigma_H, sigma_h, p_f, p0, _SYSTEMS[system], out, pf)
        return out

    def gmres_solve(self, tree: Tree, dt, rhs, x=None, system="pressure", restart=50, max_iters=1000, tol=1e-6,
                    mode="fmm", raise_on_notconv=True):
        x = torch.zeros(3 * tree.n, dtype=torch.float64, device="cuda") if x is None else x
        info = ddm_gmres_solve(self.ptr, tree.ptr, dt, rhs, x, _SYSTEMS[system], restart, max_iters, tol,
                               _MODES[mode], raise_on_notconv)
        return x, info

    def grow(self, xy, x, tips, ends, K_Ic):
        """One fracture growth step (ddm_grow)."""
        return ddm_grow(self.ptr, xy, x, tips, ends, K_Ic)

    def sif(self, tree: Tree, x, tips):
        tips = torch.as_tensor(tips, dtype=torch.int64, device="cuda").contiguous()
        KI = torch.empty(tips.numel(), dtype=torch.float64, device="cuda")
        KII = torch.empty_like(KI)
        ddm_sif(self.ptr, tree.ptr, x, tips, KI, KII)
        return KI, KII

    def batch(self, trees) -> Batch:
        return Batch(self, trees)

    def profile(self, enable=True):
        ddm_profile(self.ptr, enable)

    def profile_read(self) -> dict:
        return ddm_profile_read(self.ptr)

    def device_check(self):
        ddm_device_check(self.ptr)

    def set_wait_limit(self, polls=0):
        ddm_set_wait_limit(self.ptr, polls)

    def set_m2l_compression(self, mode=2, rank=0):
        ddm_set_m2l_compression(self.ptr, mode, rank)

    def set_history_compression(self, exact_steps=0, nodes=10, ratio=2.0):
        ddm_set_history_compression(self.ptr, exact_steps, nodes, ratio)

    def close(self):
        if self.ptr:
            ddm_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

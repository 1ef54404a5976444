"""FP64 CPU oracle for the poroelastic DDM hot path.

TEST INFRASTRUCTURE ONLY: only the test-suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  The product library
never imports, links or executes it, and it shares no code with the CUDA path.

The influence coefficients (paper Eqs. 2.3-2.5) are computed by
``ddm_oracle.c`` from their definition (Kelvin solution + moment tensor for
the drained elastic part, displacement potential + diffusion for the
poroelastic part, line-source solution for the fluid source; element
integrals by adaptive quadrature).  This module adds the plain linear algebra
on top: the dense product y = A x, the direct solve of the boundary system,
the direct time-history double sum and the Olson stress intensity factors
(Eq. 2.6).  Every function follows the plain definition with no blocking,
fusion or reordering.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libddm_oracle.so")
_lib = None
_lock = threading.Lock()

_DP = ctypes.POINTER(ctypes.c_double)
_LP = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_constants.argtypes = [_DP, _DP]
            L.orc_e1.argtypes = [ctypes.c_double]
            L.orc_e1.restype = ctypes.c_double
            L.orc_ein.argtypes = [ctypes.c_double]
            L.orc_ein.restype = ctypes.c_double
            L.orc_point_kernel.argtypes = [_DP] + [ctypes.c_double] * 8 + [ctypes.c_int, _DP]
            L.orc_element_field.argtypes = [_DP] + [ctypes.c_double] * 7 + [ctypes.c_int, _DP]
            L.orc_assemble.argtypes = [_DP, _DP, ctypes.c_int64, ctypes.c_double, _DP]
            L.orc_assemble_rows.argtypes = [_DP, _DP, ctypes.c_int64, ctypes.c_double, _LP,
                                            ctypes.c_int64, _DP]
            L.orc_field.argtypes = [_DP, _DP, ctypes.c_int64, ctypes.c_double, _DP, _DP,
                                    ctypes.c_int64, _LP, _DP]
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_DP)


def _mat(material) -> np.ndarray:
    """Material as (G, nu, nu_u, B, permeability, viscosity)."""
    if isinstance(material, dict):
        material = [material[k] for k in ("G", "nu", "nu_u", "B", "perm", "visc")]
    return np.ascontiguousarray(material, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# constants and special functions
# --------------------------------------------------------------------------
def constants(material) -> dict:
    """Biot/Rice-Cleary constants: alpha, eta, M, S, kappa, c, kpsi, lam."""
    out = np.zeros(8)
    lib().orc_constants(_d(_mat(material)), _d(out))
    keys = ("alpha", "eta", "M", "S", "kappa", "c", "kpsi", "lam")
    return dict(zip(keys, out.tolist()))


def e1(u: float) -> float:
    return float(lib().orc_e1(float(u)))


def ein(u: float) -> float:
    return float(lib().orc_ein(float(u)))


def point_kernel(material, z, t, D=(0.0, 0.0), n=(0.0, 1.0), Q=0.0, part=3) -> np.ndarray:
    """(sxx, syy, sxy, p) at offset z from a point DD vector D across normal n
    plus a point fluid source Q, switched on at time 0 and observed at t.
    part: 1 drained elastic, 2 transient, 3 both."""
    out = np.zeros(4)
    lib().orc_point_kernel(_d(_mat(material)), float(z[0]), float(z[1]), float(t), float(D[0]),
                           float(D[1]), float(n[0]), float(n[1]), float(Q), int(part), _d(out))
    return out


def element_field(material, p, y0, y1, t, self_elem=False) -> np.ndarray:
    """(3, 4): rows = unit Ds, Dn, Dq on element y0->y1; cols = sxx, syy, sxy, p
    at point p (global frame), step-on response at time t."""
    out = np.zeros(12)
    lib().orc_element_field(_d(_mat(material)), float(p[0]), float(p[1]), float(y0[0]), float(y0[1]),
                            float(y1[0]), float(y1[1]), float(t), int(bool(self_elem)), _d(out))
    return out.reshape(3, 4)


# --------------------------------------------------------------------------
# dense influence matrix and products
# --------------------------------------------------------------------------
def _xy(xy) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    assert xy.ndim == 2 and xy.shape[0] == 4
    return xy


def assemble(material, xy, t: float) -> np.ndarray:
    """Dense A(t) (3N x 3N): rows [sigma_s; sigma_n; p] at midpoints, columns
    [Ds; Dn; Dq], step-on response at time t (A(t<=0) = 0)."""
    xy = _xy(xy)
    N = xy.shape[1]
    A = np.zeros((3 * N, 3 * N))
    lib().orc_assemble(_d(_mat(material)), _d(xy), N, float(t), _d(A))
    return A


def assemble_rows(material, xy, t: float, rows) -> np.ndarray:
    """Selected rows of A(t) (row index r = comp * N + element)."""
    xy = _xy(xy)
    N = xy.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    A = np.zeros((rows.size, 3 * N))
    lib().orc_assemble_rows(_d(_mat(material)), _d(xy), N, float(t), rows.ctypes.data_as(_LP),
                            rows.size, _d(A))
    return A


def window(material, xy, t_lo: float, t_hi: float, rows=None) -> np.ndarray:
    """The time-element matrix A(t_hi) - A(t_lo) (A(0) = 0): the response at
    the observation time to a source held constant over a time element."""
    f = (lambda t: assemble(material, xy, t)) if rows is None else \
        (lambda t: assemble_rows(material, xy, t, rows))
    A = f(t_hi)
    if t_lo > 0.0:
        A = A - f(t_lo)
    return A


def matvec(material, xy, x, t_lo: float, t_hi: float, rows=None) -> np.ndarray:
    """y = (A(t_hi) - A(t_lo)) x (the plain dense product)."""
    return window(material, xy, t_lo, t_hi, rows) @ np.asarray(x, dtype=np.float64)


def field(material, xy, D, t: float, pts, on_elem=None) -> np.ndarray:
    """(npts, 4) global (sxx, syy, sxy, p) at arbitrary points."""
    xy = _xy(xy)
    N = xy.shape[1]
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = np.zeros((pts.shape[0], 4))
    oe = None if on_elem is None else np.ascontiguousarray(on_elem, dtype=np.int64)
    lib().orc_field(_d(_mat(material)), _d(xy), N, float(t), _d(D), _d(pts), pts.shape[0],
                    None if oe is None else oe.ctypes.data_as(_LP), _d(out))
    return out


# --------------------------------------------------------------------------
# boundary conditions, systems, time marching, SIF
# --------------------------------------------------------------------------
SYSTEMS = ("pressure", "impermeable", "rate")


def frames(xy):
    xy = _xy(xy)
    dx, dy = xy[2] - xy[0], xy[3] - xy[1]
    L = np.hypot(dx, dy)
    tx, ty = dx / L, dy / L
    return tx, ty, -ty, tx, L


def rhs(xy, sigma_H=0.0, sigma_h=0.0, p_f=0.0, p0=0.0, system="pressure") -> np.ndarray:
    """Known right-hand side of the first step (paper Sec. 4): far-field
    stresses (compression positive, sigma_H along x, sigma_h along y)
    resolved on each element and added to the hydraulic load.
    pressure:    [-tau_inf, -(p_f - s_nn_inf), p_f - p0]
    impermeable: [-tau_inf, -(p_f - s_nn_inf), 0]
    rate:        [-tau_inf, -(p0 - s_nn_inf),  0]   (row 2 is sigma_n + p)"""
    tx, ty, nx, ny, _ = frames(xy)
    N = tx.size
    sxx, syy = -sigma_H, -sigma_h                   # tension positive
    snn = sxx * nx * nx + syy * ny * ny             # tension positive
    tau = sxx * tx * nx + syy * ty * ny
    pf = np.broadcast_to(np.asarray(p_f, dtype=np.float64), (N,))
    b = np.zeros(3 * N)
    b[:N] = -tau
    if system == "rate":
        b[N:2 * N] = -p0 - snn
    else:
        b[N:2 * N] = -pf - snn
    if system == "pressure":
        b[2 * N:] = pf - p0
    return b


def _restrict(A, N, system):
    """Rows/columns of the boundary system and the columns moved to the RHS."""
    if system == "pressure":
        return A, None
    Ar = A[:2 * N].copy()
    if system == "rate":
        Ar[N:2 * N] += A[2 * N:]
    return Ar[:, :2 * N], Ar[:, 2 * N:]


def solve(A, b, N, system="pressure", Dq=None) -> np.ndarray:
    """Solve the boundary system with a direct LU solve (numpy).  Returns the
    full 3N vector [Ds, Dn, Dq] (Dq prescribed for the 2N systems).  b holds
    row values [sigma_s, sigma_n, p]; the RATE system's second row is
    sigma_n + p, so its right-hand side is b_n + b_p (b_p is zero for a
    first step and carries the pressure part of a subtracted history)."""
    if system == "pressure":
        return np.linalg.solve(A, b)
    Asub, Aq = _restrict(A, N, system)
    Dq = np.zeros(N) if Dq is None else np.broadcast_to(np.asarray(Dq, float), (N,))
    bb = b[:2 * N].copy()
    if system == "rate":
        bb[N:] = b[N:2 * N] + b[2 * N:]
    bb = bb - Aq @ Dq
    x = np.linalg.solve(Asub, bb)
    return np.concatenate([x, Dq])


def history(material, xy, hist, times, rows=None) -> np.ndarray:
    """Direct time-history double sum of Eqs. (2.3)-(2.5):
    sum_{eta=1}^{H} [A(t_{H+1} - t_{eta-1}) - A(t_{H+1} - t_eta)] D^eta
    with hist[eta-1] = D^eta and times = (t_0, ..., t_{H+1}).  The caller
    subtracts it from the right-hand side of step H+1."""
    hist = np.atleast_2d(np.asarray(hist, dtype=np.float64))
    H = hist.shape[0]
    times = np.asarray(times, dtype=np.float64)
    assert times.size == H + 2
    th = times[-1]
    out = 0.0
    for eta in range(1, H + 1):
        out = out + matvec(material, xy, hist[eta - 1], th - times[eta], th - times[eta - 1], rows)
    return out


def march(material, xy, times, b_steps, system="pressure", Dq_steps=None) -> np.ndarray:
    """Time marching (paper Sec. 4 algorithm): for each step, subtract the
    history of all previous steps from the known RHS and solve.  Returns the
    solutions D^1..D^H (H x 3N).  Uses dense matrices and direct solves."""
    xy = _xy(xy)
    N = xy.shape[1]
    times = np.asarray(times, dtype=np.float64)
    H = times.size - 1
    cache = {}

    def A_at(t):
        key = round(float(t), 12)
        if key not in cache:
            cache[key] = assemble(material, xy, t)
        return cache[key]

    sols = []
    for h in range(1, H + 1):
        th = times[h]
        b = np.array(b_steps[h - 1], dtype=np.float64)
        for eta in range(1, h):
            b -= (A_at(th - times[eta - 1]) - A_at(th - times[eta])) @ sols[eta - 1]
        Dq = None if Dq_steps is None else Dq_steps[h - 1]
        sols.append(solve(A_at(th - times[h - 1]), b, N, system, Dq))
    return np.array(sols)


def sif(material, xy, D, tip_elems, drained=True):
    """Olson's tip-element formula (paper Eq. 2.6):
    K = 0.806 E / (4 (1 - nu^2)) sqrt(pi / (2 a)) D, with a the half-length
    of the tip element (a reading) and (E, nu) drained unless told otherwise.
    Returns (K_I, K_II) arrays for the given tip elements."""
    m = _mat(material)
    G, nu = m[0], (m[1] if drained else m[2])
    E = 2.0 * G * (1.0 + nu)
    _, _, _, _, L = frames(xy)
    N = L.size
    tip = np.asarray(tip_elems, dtype=np.int64)
    a = 0.5 * L[tip]
    f = 0.806 * E / (4.0 * (1.0 - nu * nu)) * np.sqrt(np.pi / (2.0 * a))
    D = np.asarray(D)
    return f * D[N + tip], f * D[tip]


def kink(KI, KII):
    """Maximum tangential stress criterion (Erdogan and Sih; the paper's
    propagation check in the Sec. 4 algorithm names no criterion, this is
    the reading): in the crack-tip frame the hoop stress ahead of the tip at
    angle theta is proportional to
        s(theta) = cos(theta/2) (K_I cos^2(theta/2) - 1.5 K_II sin(theta));
    its maximiser theta_c solves K_I sin(theta) + K_II (3 cos(theta) - 1) = 0,
        theta_c = 2 atan((K_I - sqrt(K_I^2 + 8 K_II^2)) / (4 K_II))  (0 if K_II = 0),
    and K_eq = s(theta_c).  Returns (theta_c, K_eq) arrays."""
    KI = np.asarray(KI, dtype=np.float64)
    KII = np.asarray(KII, dtype=np.float64)
    safe = np.where(KII != 0.0, KII, 1.0)
    th = np.where(KII != 0.0, 2.0 * np.arctan((KI - np.sqrt(KI * KI + 8.0 * KII * KII)) / (4.0 * safe)), 0.0)
    c = np.cos(0.5 * th)
    return th, c * (KI * c * c - 1.5 * KII * np.sin(th))


def grow(material, xy, D, tips, ends, K_Ic):
    """One growth step (reading of the paper's propagation check, Sec. 4):
    for every tip (element tips[i], its end ends[i] = 0 for (x0, y0), 1 for
    (x1, y1)), K_I and K_II by Olson's formula (sif, drained), taken in the
    crack-tip frame x = outward tangent, y = x turned by +90 degrees (the
    element frame's signs at either end, as the opening keeps its sign),
    theta and K_eq by kink(); a tip with K_I > 0 and K_eq >= K_Ic grows by an
    element as long as its tip element, from the tip along x turned by
    theta.  Returns (grown xy 4 x (N + grown), tips, ends, theta, K_eq):
    the old elements first, the new ones in tip order, a grown tip moved to
    its new element's end 1."""
    xy = _xy(xy)
    N = xy.shape[1]
    tips = np.asarray(tips, dtype=np.int64).copy()
    ends = np.asarray(ends, dtype=np.int64).copy()
    KI, KII = sif(material, xy, D, tips)
    th, keq = kink(KI, KII)
    new = []
    for i, e in enumerate(tips):
        a, b = xy[:2, e], xy[2:, e]
        L = np.hypot(*(b - a))
        x_dir = (b - a) / L if ends[i] == 1 else (a - b) / L
        y_dir = np.array([-x_dir[1], x_dir[0]])
        p = b if ends[i] == 1 else a
        if KI[i] > 0.0 and keq[i] >= K_Ic:
            d = np.cos(th[i]) * x_dir + np.sin(th[i]) * y_dir
            new.append(np.concatenate([p, p + L * d]))
            tips[i] = N + len(new) - 1
            ends[i] = 1
    if new:
        xy = np.concatenate([xy, np.array(new).T], axis=1)
    return xy, tips, ends, th, keq

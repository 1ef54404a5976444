"""The benchmark configurations against the FP64 oracle and the closed forms.

- Single pressurised crack (200 elements, a = 1 m, p = 1 MPa): FP64 dense
  product (exact element integrals) and GMRES to 1e-10, in the drained and
  undrained limits, against the oracle's direct solution and against the
  Sneddon opening and K_I = p sqrt(pi a) (paper Eq. 2.6).
- Stress intensity factors of a GMRES solution against Eq. 2.6 applied to
  the oracle's direct solution (not to the GPU's own vector).
- Horizontal-well time march (paper Sec. 5 example; RATE system, 60 s
  steps, the history of all previous steps subtracted at every step):
  a reduced instance (10 x 40 elements, 100 steps) against the oracle's
  full march stored in tests/golden/well_march_10x40.json, and the full
  size (10 x 2,000 elements, 100 steps) with the residual of the exact
  operator on sampled rows."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev, small_random_set

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)


def k_close(got, ref, rel=1e-3, floor=0.1):
    """Per-tip relative error of stress intensity factors, each measured
    against max(|K_ref|, floor * max |K_ref| over the tips)."""
    got, ref = np.asarray(got), np.asarray(ref)
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max())
    return np.max(np.abs(got - ref) / scale) < rel


# ----------------------------------------------------------------------------
# single crack, FP64 dense, tol 1e-10
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("limit", ["drained", "undrained"])
def test_single_crack_fp64_dense_sneddon(ctx, limit):
    N, a, p = 200, 1.0, 1e6
    dt, nu_eff = (1e12, MAT[1]) if limit == "drained" else (1e-4, MAT[2])
    xy = inputs.single_crack(N, a)
    xm = 0.5 * (xy[0] + xy[2])
    tree = ctx.build_tree(dev(xy))
    b = ctx.rhs(tree, p_f=p, system="impermeable")
    x, info = ctx.gmres_solve(tree, dt, b, system="impermeable", tol=1e-10, mode="dense+precise")
    assert info["converged"] and info["rel_residual"] < 1e-10
    xs = x.cpu().numpy()
    ref = oracle.solve(oracle.assemble(MAT, xy, dt), oracle.rhs(xy, p_f=p, system="impermeable"), N, "impermeable")
    assert block_rel_err(xs, ref, N, blocks=2) < 1e-6
    Dn = xs[N:2 * N]
    w = 2 * (1 - nu_eff) * p / MAT[0] * np.sqrt(a * a - xm ** 2)
    mid = np.abs(xm) <= 0.8 * a
    assert np.max(np.abs(Dn[mid] / w[mid] - 1)) < 0.01
    tips = [0, N - 1]
    KI, _ = ctx.sif(tree, x, tips)
    KI = KI.cpu().numpy()
    rI, _ = oracle.sif(MAT, xy, ref, tips)
    assert np.max(np.abs(KI / rI - 1)) < 1e-6
    if limit == "drained":
        assert np.all(np.abs(KI / (p * math.sqrt(math.pi * a)) - 1) < 0.02)
    else:   # the library's K uses drained (E, nu): K = p sqrt(pi a) (1 - nu_u) / (1 - nu)
        assert np.all(np.abs(KI / (p * math.sqrt(math.pi * a) * (1 - MAT[2]) / (1 - MAT[1])) - 1) < 0.02)


def test_single_crack_pressure_system_fp64(ctx):
    """Full 3N system (D_q unknown, pressure row) at the nominal 10 s step."""
    N = 200
    xy = inputs.single_crack(N, 1.0)
    tree = ctx.build_tree(dev(xy))
    b = ctx.rhs(tree, p_f=1e6, p0=2e5, system="pressure")
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-10, mode="dense+precise")
    assert info["converged"]
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), oracle.rhs(xy, p_f=1e6, p0=2e5, system="pressure"), N)
    assert block_rel_err(x.cpu().numpy(), ref, N) < 1e-6


# ----------------------------------------------------------------------------
# SIFs of a solve against Eq. 2.6 on the oracle's solution
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fmm", "dense"])
def test_sif_of_solve_matches_oracle_solution(ctx, mode):
    xy, segs = small_random_set()
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    loads = dict(sigma_H=30e6, sigma_h=25e6, p_f=10e6, p0=0.0)
    b = ctx.rhs(tree, system="pressure", **loads)
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-6, mode=mode)
    assert info["converged"]
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), oracle.rhs(xy, system="pressure", **loads), N)
    tips = inputs.tips_of(segs)
    KI, KII = ctx.sif(tree, x, tips)
    rI, rII = oracle.sif(MAT, xy, ref, tips)
    assert k_close(KI.cpu().numpy(), rI)
    assert k_close(KII.cpu().numpy(), rII)
    assert block_rel_err(x.cpu().numpy(), ref, N) < 1e-3


# ----------------------------------------------------------------------------
# horizontal-well time march
# ----------------------------------------------------------------------------
def march(ctx, tree, N, steps, half_length, keep=(), tol=1e-6):
    """Paper Sec. 4 time marching on the GPU: for each step subtract the
    history of all previous steps (ddm_history_apply) from the known
    right-hand side and solve the RATE system (x0 = previous solution, the
    fluid source prescribed).  Returns the device history (steps x 3N) and
    the GMRES infos."""
    hist = torch.zeros(steps, 3 * N, dtype=torch.float64, device="cuda")
    b0 = ctx.rhs(tree, system="rate", **inputs.WELL_LOADS)
    times = [inputs.WELL_DT * k for k in range(steps + 1)]
    x = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    x[2 * N:] = inputs.well_source(half_length)
    infos = []
    for h in range(1, steps + 1):
        b = b0.clone()
        if h > 1:
            ctx.history_apply(tree, hist[:h - 1], times[:h + 1], b)
        x, info = ctx.gmres_solve(tree, inputs.WELL_DT, b, x, system="rate", tol=tol)
        hist[h - 1] = x
        infos.append(info)
    return hist, infos


def test_well_march_reduced_matches_oracle(ctx):
    g = json.load(open(os.path.join(HERE, "golden", "well_march_10x40.json")))
    xy, segs = inputs.parallel_fractures(n_frac=g["n_frac"], spacing=g["spacing"], half_length=g["half_length"],
                                         elems=g["elems"])
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    hist, infos = march(ctx, tree, N, g["steps"], g["half_length"])
    assert all(i["converged"] for i in infos)
    H = hist.cpu().numpy()
    for h, ref in g["D"].items():
        got = H[int(h) - 1]
        assert block_rel_err(got, np.asarray(ref), N, blocks=2) < 1e-3, h
    tips = np.asarray(g["tips"])
    for h in g["KI"]:
        KI, KII = ctx.sif(tree, hist[int(h) - 1].contiguous(), tips)
        assert k_close(KI.cpu().numpy(), g["KI"][h]), h
        assert k_close(KII.cpu().numpy(), g["KII"][h]), h


def test_well_march_full_size_residual_sampled(ctx):
    """10 x 2,000 elements, 100 steps: every step converges, and at steps
    1, 2 and 5 the GPU solutions satisfy the exact equations (oracle rows of
    every time element, history included) at the tips and centres of the
    third and fifth fractures.  Residuals are measured against the system's
    right-hand side with the prescribed source moved to it (as GMRES
    measures them).  With 2,000 elements per fracture the FP32 products
    floor GMRES near 1.5e-5 of that right-hand side at the first step and
    near 1.4e-4 from about step 40 on, once the opening has grown smooth and
    the element contributions cancel, so the march runs to 3e-4; the exact
    residual (history included) stays within 1e-2 of it.  The reduced
    instance above is held to 1e-3 against the oracle's march."""
    half = 100.0
    xy, segs = inputs.parallel_fractures(n_frac=10, spacing=20.0, half_length=half, elems=2000)
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    steps = 100
    hist, infos = march(ctx, tree, N, steps, half, tol=3e-4)
    assert all(i["converged"] for i in infos)
    H = hist[:5].cpu().numpy()
    el = np.array([2 * 2000, 2 * 2000 + 1000, 3 * 2000 - 1, 4 * 2000, 4 * 2000 + 1000, 5 * 2000 - 1])
    rows = np.concatenate([el + c * N for c in range(3)])
    k = el.size
    b = oracle.rhs(xy, system="rate", **inputs.WELL_LOADS)
    bsys = np.concatenate([b[el], b[N + el]])
    A = {}
    dt = inputs.WELL_DT
    for h in (1, 2, 5):
        # rows of sum_eta [A(t_h - t_{eta-1}) - A(t_h - t_eta)] D^eta, A(0) = 0
        y = np.zeros(3 * k)
        for eta in range(1, h + 1):
            for lag, sgn in ((h - eta + 1, 1.0), (h - eta, -1.0)):
                if lag == 0:
                    continue
                if lag not in A:
                    A[lag] = oracle.assemble_rows(MAT, xy, lag * dt, rows)
                y += sgn * (A[lag] @ H[eta - 1])
        res = np.concatenate([y[:k], y[k:2 * k] + y[2 * k:]]) - bsys
        yq = A[1][:, 2 * N:] @ H[h - 1][2 * N:]           # the current step's prescribed source
        scale = np.abs(bsys - np.concatenate([yq[:k], yq[k:2 * k] + yq[2 * k:]])).max()
        assert np.abs(res).max() < 1e-2 * scale, h

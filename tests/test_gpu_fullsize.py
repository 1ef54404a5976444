"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (n_cheb = 8, leaf 32): sampled rows that the FP64 oracle computes one
by one (all N sources each), and the GMRES residual checked on sampled rows
of the exact operator."""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)


@pytest.fixture(scope="module")
def random_set():
    xy, segs = inputs.random_fractures()
    return xy, segs


def sampled_rows(N, k, seed):
    rng = np.random.default_rng(seed)
    el = np.sort(rng.choice(N, k, replace=False))
    return el, np.concatenate([el + b * N for b in range(3)])


def test_random_fractures_products_sampled(ctx, random_set):
    xy, _ = random_set
    N = xy.shape[1]
    tree = ctx.build_tree(torch.as_tensor(xy, device="cuda"))
    x = inputs.unknowns(N, seed=99)
    dx = torch.as_tensor(x, device="cuda")
    el, rows = sampled_rows(N, 9, 5)
    A = oracle.assemble_rows(MAT, xy, 10.0, rows)
    ref = A @ x
    k = el.size
    for mode, tol in (("fmm", 1e-4), ("dense", 2e-5)):
        y = ctx.matvec(tree, dx, 0.0, 10.0, mode=mode).cpu().numpy()[rows]
        for b in range(3):
            r = ref[b * k:(b + 1) * k]
            assert np.abs(y[b * k:(b + 1) * k] - r).max() < tol * np.abs(r).max(), (mode, b)


def test_random_fractures_fmm_matches_dense_everywhere(ctx, random_set):
    """Every row: FMM (n = 8) against the on-the-fly dense product."""
    xy, _ = random_set
    N = xy.shape[1]
    tree = ctx.build_tree(torch.as_tensor(xy, device="cuda"))
    dx = torch.as_tensor(inputs.unknowns(N, seed=98), device="cuda")
    yf = ctx.matvec(tree, dx, 0.0, 10.0, mode="fmm").cpu().numpy()
    yd = ctx.matvec(tree, dx, 0.0, 10.0, mode="dense").cpu().numpy()
    for b in range(3):
        assert np.abs(yf[b * N:(b + 1) * N] - yd[b * N:(b + 1) * N]).max() < 1e-4 * np.abs(yd[b * N:(b + 1) * N]).max()


def test_random_fractures_gmres_residual_sampled(ctx, random_set):
    xy, segs = random_set
    N = xy.shape[1]
    tree = ctx.build_tree(torch.as_tensor(xy, device="cuda"))
    loads = dict(sigma_H=30e6, sigma_h=25e6, p_f=10e6, p0=0.0)
    b = ctx.rhs(tree, system="pressure", **loads)
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-5)
    assert info["converged"]
    xs = x.cpu().numpy()
    el, rows = sampled_rows(N, 9, 6)
    A = oracle.assemble_rows(MAT, xy, 10.0, rows)
    bref = oracle.rhs(xy, system="pressure", **loads)
    res = A @ xs - bref[rows]
    assert np.abs(res).max() < 1e-3 * np.abs(bref).max()


def test_parallel_fractures_history_sampled(ctx):
    """History double sum on the horizontal-well geometry (10 fractures,
    reduced to 400 elements each), 6 past steps of 60 s."""
    xy, _ = inputs.parallel_fractures(n_frac=10, spacing=20.0, half_length=100.0, elems=400)
    N = xy.shape[1]
    tree = ctx.build_tree(torch.as_tensor(xy, device="cuda"))
    H = 6
    times = [60.0 * k for k in range(H + 2)]
    hist = np.stack([inputs.unknowns(N, seed=40 + k) for k in range(H)])
    rhs0 = np.zeros(3 * N)
    got = -ctx.history_apply(tree, torch.as_tensor(hist, device="cuda"), times,
                             torch.as_tensor(rhs0, device="cuda")).cpu().numpy()
    el, rows = sampled_rows(N, 12, 8)
    ref = oracle.history(MAT, xy, hist, times, rows=rows)
    k = el.size
    for b in range(3):
        r = ref[b * k:(b + 1) * k]
        assert np.abs(got[rows][b * k:(b + 1) * k] - r).max() < 2e-4 * np.abs(r).max(), b

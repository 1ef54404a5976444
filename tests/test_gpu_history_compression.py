"""Time-compressed history sum (ddm_set_history_compression): the older past
steps interpolated in log time over geometric blocks, the recent ones exact.

- Against the FP64 oracle's exact double sum (paper Sec. 4 time marching)
  on a small geometry, 40 constant steps of 60 s, random past solutions.
- Against the library's exact sum on 10 x 40 parallel fractures (the
  horizontal-well layout, reduced), 100 steps: the error falls with the
  node count, and the number of FMM products is exact_steps + (nodes - 1)
  per block instead of one per past step.
- Growing steps (x1.05 per step): the block intervals widen to the windows.
- Few past steps (H <= exact_steps): the exact sum.
- Bad settings are rejected."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context, DDMError

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
DT = 60.0


def random_history(N, H, seed):
    return np.stack([inputs.unknowns(N, seed=seed + k) for k in range(H)])


def history(ctx, tree, hist, times):
    rhs = torch.zeros(hist.shape[1], dtype=torch.float64, device="cuda")
    ctx.history_apply(tree, dev(hist), list(times), rhs)
    return -rhs.cpu().numpy()                     # the sum itself (the call subtracts it)


def products(ctx, fn):
    ctx.profile_read()
    fn()
    return ctx.profile_read()["prep"][1]


def test_compressed_history_matches_oracle():
    xy, _ = inputs.parallel_fractures(n_frac=2, spacing=20.0, half_length=15.0, elems=15)
    N = xy.shape[1]
    H = 40
    hist = random_history(N, H, seed=300)
    times = DT * np.arange(H + 2)
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=4)
    tree = ctx.build_tree(dev(xy))
    ctx.set_history_compression(4, 10, 2.0)
    got = history(ctx, tree, hist, times)
    ref = oracle.history(MAT, xy, hist, times)
    e = block_rel_err(got, ref, N)
    print(f"compressed vs oracle: {e:.2e}")
    assert e < 5e-5
    ctx.device_check()


@pytest.fixture(scope="module")
def well():
    xy, _ = inputs.parallel_fractures(n_frac=10, spacing=20.0, half_length=100.0, elems=40)
    return xy


def test_compressed_history_vs_exact_sum(well):
    xy = well
    N = xy.shape[1]
    H = 100
    hist = random_history(N, H, seed=400)
    times = DT * np.arange(H + 2)
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    tree = ctx.build_tree(dev(xy))
    ref = history(ctx, tree, hist, times)
    errs = {}
    for p in (6, 8, 10, 12):
        ctx.set_history_compression(8, p, 2.0)
        got = history(ctx, tree, hist, times)
        errs[p] = block_rel_err(got, ref, N)
        # blocks of lo = t_obs - t_eta: [9, 18), [18, 36), [36, 72), [72, 144) steps
        n = products(ctx, lambda: history(ctx, tree, hist, times))
        print(f"nodes {p}: {n} products (exact {H}), error vs exact sum {errs[p]:.2e}")
        assert n == 8 + 4 * (p - 1)
    assert errs[10] < 2e-5 and errs[12] < 2e-5
    assert errs[8] < errs[6]
    # the exact sum again with compression off
    ctx.set_history_compression(0)
    assert products(ctx, lambda: history(ctx, tree, hist, times)) == H
    ctx.device_check()


def test_compressed_history_growing_steps(well):
    xy = well
    N = xy.shape[1]
    H = 60
    hist = random_history(N, H, seed=500)
    steps = DT * 1.05 ** np.arange(H + 1)
    times = np.concatenate([[0.0], np.cumsum(steps)])
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    tree = ctx.build_tree(dev(xy))
    ref = history(ctx, tree, hist, times)
    ctx.set_history_compression(8, 10, 2.0)
    got = history(ctx, tree, hist, times)
    e = block_rel_err(got, ref, N)
    print(f"growing steps: error vs exact sum {e:.2e}")
    assert e < 2e-5
    ctx.device_check()


def test_few_steps_take_the_exact_sum(well):
    xy = well
    N = xy.shape[1]
    H = 8
    hist = random_history(N, H, seed=600)
    times = DT * np.arange(H + 2)
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    tree = ctx.build_tree(dev(xy))
    ref = history(ctx, tree, hist, times)
    ctx.set_history_compression(8, 10, 2.0)
    assert products(ctx, lambda: history(ctx, tree, hist, times)) == H
    assert block_rel_err(history(ctx, tree, hist, times), ref, N) < 1e-6


def test_bad_settings_rejected():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    for args in ((-1, 10, 2.0), (8, 1, 2.0), (8, 17, 2.0), (8, 10, 1.2), (8, 10, 20.0), (8, 10, math.nan)):
        with pytest.raises(DDMError):
            ctx.set_history_compression(*args)
    ctx.set_history_compression(0)                # off: any nodes and ratio

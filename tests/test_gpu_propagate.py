"""Fracture growth step (ddm_grow; the propagation check of the paper's
Sec. 4 time-marching algorithm with the maximum tangential stress
criterion as the reading).

- The GPU step against oracle.grow on the same solution vector: growth
  flags, updated tips, kink angles, K_eq and the grown geometry.
- A growth loop (solve -> grow -> rebuild the tree) of a pressurised crack
  at 45 degrees under sigma_H > sigma_h: the first kink turns it toward the
  x axis and it stays near that direction, and every step's GPU solve
  matches the oracle's direct solve on the grown geometry.
- No tips, and a toughness no tip reaches: the geometry is unchanged."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev, small_random_set

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
LOADS = dict(sigma_H=20e6, sigma_h=10e6, p_f=25e6, p0=0.0)
DT = 1e12                     # drained


def inclined(N=40, a=1.0, angle=math.pi / 4):
    xy = inputs.single_crack(N, a)
    c, s = math.cos(angle), math.sin(angle)
    rot = np.array([[c, -s], [s, c]])
    return np.vstack([rot @ xy[:2], rot @ xy[2:]])


def solve(ctx, xy):
    tree = ctx.build_tree(dev(xy))
    b = ctx.rhs(tree, system="impermeable", **LOADS)
    x, info = ctx.gmres_solve(tree, DT, b, system="impermeable", tol=1e-8, mode="fmm")
    assert info["converged"]
    return tree, x


def test_grow_matches_oracle_step():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=8)
    xy_a = inclined()
    xy_b, segs = small_random_set(n_frac=6, box=12.0, elems=20, seed=31)
    for xy, tips, ends in ((xy_a, [0, 39], [0, 1]),
                           (xy_b, list(inputs.tips_of(segs)), [0, 1] * len(segs))):
        N = xy.shape[1]
        tree, x = solve(ctx, xy)
        t = torch.tensor(tips, dtype=torch.int64, device="cuda")
        e = torch.tensor(ends, dtype=torch.int32, device="cuda")
        xs = x.cpu().numpy()
        KI, KII = oracle.sif(MAT, xy, xs, tips)
        v = np.sort(oracle.kink(KI, KII)[1])
        K_Ic = 0.5 * (v[len(v) // 2 - 1] + v[len(v) // 2])    # half of the tips grow, none at the bound
        g, th, keq = ctx.grow(dev(xy), x, t, e, K_Ic)
        rg, rt, re_, rth, rkeq = oracle.grow(MAT, xy, xs, tips, ends, K_Ic)
        assert g.shape == rg.shape and g.shape[1] > N
        assert np.array_equal(t.cpu().numpy(), rt) and np.array_equal(e.cpu().numpy(), re_)
        assert np.allclose(th.cpu().numpy(), rth, rtol=0, atol=1e-12)
        assert np.allclose(keq.cpu().numpy(), rkeq, rtol=1e-12, atol=0)
        assert np.allclose(g.cpu().numpy(), rg, rtol=0, atol=1e-12)
    ctx.device_check()


def test_growth_loop_turns_toward_sigma_H():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=8)
    xy = inclined()
    tips = torch.tensor([0, xy.shape[1] - 1], dtype=torch.int64, device="cuda")
    ends = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    slopes = []
    for step in range(6):
        N = xy.shape[1]
        tree, x = solve(ctx, xy)
        ref = oracle.solve(oracle.assemble(MAT, xy, DT), oracle.rhs(xy, system="impermeable", **LOADS), N,
                           "impermeable")
        assert block_rel_err(x.cpu().numpy(), ref, N, blocks=2) < 1e-3, step
        g, th, keq = ctx.grow(dev(xy), x, tips, ends, 0.0)
        g = g.cpu().numpy()
        assert g.shape[1] == N + 2, step                          # both tips grow (K_Ic = 0)
        d = g[2:, N + 1] - g[:2, N + 1]                            # the new element at the upper tip
        slopes.append(abs(d[1] / d[0]))
        xy = np.ascontiguousarray(g)
    print("slopes of the new tip elements:", ["%.3f" % s for s in slopes])
    assert slopes[0] < 0.9 and slopes[-1] <= slopes[0] + 1e-9
    ctx.device_check()


def test_no_growth_cases():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=8)
    xy = inclined()
    N = xy.shape[1]
    tree, x = solve(ctx, xy)
    t = torch.tensor([0, N - 1], dtype=torch.int64, device="cuda")
    e = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    g, th, keq = ctx.grow(dev(xy), x, t, e, 1e30)
    assert g.shape[1] == N and np.array_equal(g.cpu().numpy(), xy)
    assert t.cpu().tolist() == [0, N - 1]
    g, _, _ = ctx.grow(dev(xy), x, torch.empty(0, dtype=torch.int64, device="cuda"),
                       torch.empty(0, dtype=torch.int32, device="cuda"), 0.0)
    assert g.shape[1] == N and np.array_equal(g.cpu().numpy(), xy)


def test_growth_inside_time_marching():
    """Growth inside the time march of paper Sec. 4: after each 10 s step
    the tips grow (K_Ic = 0) and the next step's history covers the grown
    geometry, the new elements with zero past displacement discontinuity
    (they did not exist).  Every step's GPU solution against the oracle's
    direct solve of that step: A(dt) on the current geometry, the right-hand
    side minus the oracle's history sum of the zero-padded past solutions."""
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=8)
    xy = inclined(N=24)
    dt = 10.0
    tips = torch.tensor([0, xy.shape[1] - 1], dtype=torch.int64, device="cuda")
    ends = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    past = []                                            # host solutions, each at its own N
    for h in range(1, 5):
        N = xy.shape[1]
        hist = np.zeros((len(past), 3 * N))
        for k, D in enumerate(past):                     # pad every block of 3 with zeros for new elements
            n0 = D.size // 3
            for b in range(3):
                hist[k, b * N:b * N + n0] = D[b * n0:(b + 1) * n0]
        times = [dt * k for k in range(h + 1)]
        tree = ctx.build_tree(dev(xy))
        rhs = ctx.rhs(tree, system="pressure", **LOADS)
        if past:
            ctx.history_apply(tree, dev(hist), times, rhs)
        x, info = ctx.gmres_solve(tree, dt, rhs, system="pressure", tol=1e-8, mode="fmm")
        assert info["converged"], h
        b = oracle.rhs(xy, system="pressure", **LOADS)
        if past:
            b = b - oracle.history(MAT, xy, hist, times)
        ref = oracle.solve(oracle.assemble(MAT, xy, dt), b, N)
        assert block_rel_err(x.cpu().numpy(), ref, N) < 1e-3, h
        past.append(x.cpu().numpy())
        g, _, _ = ctx.grow(dev(xy), x, tips, ends, 0.0)
        xy = np.ascontiguousarray(g.cpu().numpy())
        assert xy.shape[1] == N + 2
    ctx.device_check()

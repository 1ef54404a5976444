"""Batched uneven problems (one graph launch per product, lockstep GMRES):
every problem's result in the batch equals its result alone, and the
solutions match the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()


def problems():
    out = [inputs.single_crack(64, 0.5)]
    for k, (nf, el, box) in enumerate([(3, 20, 8.0), (8, 30, 15.0), (20, 25, 25.0), (1, 150, 5.0)]):
        segs = inputs.random_fracture_segments(nf, box, 1.0, min(6.0, box / 2), el, seed=100 + k)
        out.append(inputs.assemble(segs))
    return out


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)


def test_batch_product_equals_alone(ctx):
    geos = problems()
    trees = [ctx.build_tree(dev(g)) for g in geos]
    xs = [inputs.unknowns(g.shape[1], seed=7 + i) for i, g in enumerate(geos)]
    batch = ctx.batch(trees)
    x = dev(np.concatenate(xs))
    for mode in ("fmm", "dense"):
        y = batch.matvec(x, 10.0, mode=mode).cpu().numpy()
        y2 = batch.matvec(x, 10.0, mode=mode).cpu().numpy()       # graph replay
        for i, (t, g) in enumerate(zip(trees, geos)):
            n = g.shape[1]
            alone = ctx.matvec(t, dev(xs[i]), 0.0, 10.0, mode=mode).cpu().numpy()
            seg = y[batch.offsets[i]:batch.offsets[i + 1]]
            assert block_rel_err(seg, alone, n) < 1e-5
            assert block_rel_err(y2[batch.offsets[i]:batch.offsets[i + 1]], alone, n) < 1e-5


@pytest.mark.parametrize("system", ["pressure", "impermeable"])
def test_batch_gmres_equals_alone_and_oracle(ctx, system):
    geos = problems()
    trees = [ctx.build_tree(dev(g)) for g in geos]
    rhs = [ctx.rhs(t, sigma_H=3e6, sigma_h=2e6, p_f=5e6, system=system) for t in trees]
    batch = ctx.batch(trees)
    x, infos = batch.gmres_solve(10.0, torch.cat(rhs), system=system, tol=1e-5)
    assert all(i["converged"] for i in infos)
    xs = x.cpu().numpy()
    nb = 3 if system == "pressure" else 2
    for i, (t, g) in enumerate(zip(trees, geos)):
        n = g.shape[1]
        seg = xs[batch.offsets[i]:batch.offsets[i + 1]]
        alone, info = ctx.gmres_solve(t, 10.0, rhs[i], system=system, tol=1e-5)
        assert block_rel_err(seg, alone.cpu().numpy(), n, nb) < 2e-4
        if n <= 200:
            ref = oracle.solve(oracle.assemble(MAT, g, 10.0),
                               oracle.rhs(g, sigma_H=3e6, sigma_h=2e6, p_f=5e6, system=system), n, system)
            assert block_rel_err(seg, ref, n, nb) < 1e-3


def test_batch_mixed_orders_equals_alone(ctx):
    """Trees with their own Chebyshev orders and leaf sizes in one batch:
    the batched product (one work list per order) equals every problem's
    product alone, and a tree built with order 12 gives the product of a
    context of order 12."""
    geos = problems()
    prm = [(6, 16), (8, 32), (12, 16), (8, 16), (10, 64)]
    trees = [ctx.build_tree(dev(g), n_cheb=o, leaf_size=lf) for g, (o, lf) in zip(geos, prm)]
    xs = [inputs.unknowns(g.shape[1], seed=17 + i) for i, g in enumerate(geos)]
    batch = ctx.batch(trees)
    y = batch.matvec(dev(np.concatenate(xs)), 10.0, mode="fmm").cpu().numpy()
    for i, (t, g) in enumerate(zip(trees, geos)):
        alone = ctx.matvec(t, dev(xs[i]), 0.0, 10.0, mode="fmm").cpu().numpy()
        assert block_rel_err(y[batch.offsets[i]:batch.offsets[i + 1]], alone, g.shape[1]) < 1e-5
    c12 = Context(inputs.MATERIAL, n_cheb=12, leaf_size=16)
    t12 = c12.build_tree(dev(geos[2]))
    ref12 = c12.matvec(t12, dev(xs[2]), 0.0, 10.0, mode="fmm").cpu().numpy()
    got12 = ctx.matvec(trees[2], dev(xs[2]), 0.0, 10.0, mode="fmm").cpu().numpy()
    assert block_rel_err(got12, ref12, geos[2].shape[1]) < 1e-5


def test_autotune_meets_bound_and_oracle(ctx):
    """The tuner's choice (order, leaf size, uniform or adaptive tree) for a
    random fracture set meets its error bound against the dense product, and
    its product matches the FP64 oracle."""
    segs = inputs.random_fracture_segments(30, 40.0, 2.0, 8.0, 40, seed=123)
    g = inputs.assemble(segs)
    n = g.shape[1]
    x = inputs.unknowns(n, seed=5)
    best = ctx.autotune(dev(g), dev(x), 10.0, orders=[4, 6, 8], leaves=[16, 32], max_rel_err=1e-4)
    assert best["n_cheb"] in (4, 6, 8) and best["leaf_size"] in (16, 32)
    assert best["err"] <= 1e-4 and best["ms"] > 0
    assert best["adaptive"] in (False, True)
    t = ctx.build_tree(dev(g), n_cheb=best["n_cheb"], leaf_size=best["leaf_size"], adaptive=best["adaptive"])
    y = ctx.matvec(t, dev(x), 0.0, 10.0, mode="fmm").cpu().numpy()
    rows = np.arange(0, n, 97)
    el_rows = np.concatenate([rows + b * n for b in range(3)])
    ref = oracle.matvec(MAT, g, x, 0.0, 10.0, rows=el_rows)
    k = rows.size
    for b in range(3):
        r = ref[b * k:(b + 1) * k]
        assert np.abs(y[el_rows][b * k:(b + 1) * k] - r).max() < 2e-4 * np.abs(r).max()

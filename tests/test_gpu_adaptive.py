"""Adaptive quadtree (paper Sec. 3.1: every cell holding more than leaf_size
elements is split into four, recursively, so leaves sit at different levels)
on strongly clustered fracture sets.

- Products against the FP64 oracle on a small clustered set (leaves on
  levels 2 to 8), in several time windows including a history window, and
  the solve against the oracle's direct solve.
- A leaf above level 2 (a lone crack far from a refined swarm): it has no
  far field and interacts directly with everything.
- A leaf with more than 32 direct-interaction records (graded refinement
  towards a point): the near kernels walk the records in chunks.
- 10,000 clustered elements against the GPU dense product at n = 8 and 12:
  the adaptive tree refines the swarms below the depth to which the
  longest cracks cap a uniform tree, so it has fewer direct pairs.
- Batched products of adaptive trees equal their single products."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
FMM_TOL = 2e-4                # as the uniform tree's FMM parity bar (n = 8)


def small_clustered():
    xy, _ = inputs.clustered_fractures(n_clusters=2, per_cluster=25, elems_small=8, n_sparse=4, box=120.0,
                                       elems_sparse=30, cluster_box=6.0)
    return xy


def graded(n_shell=11, per=8, r0=0.01):
    """An 8 x 8 grid of tiny cracks in an r0 square at the origin, and
    n_shell rings of per short cracks at radii 2 r0 2^k, each crack 1/8 of
    its radius long (two elements): the tree refines geometrically towards
    the origin, so the deepest leaf touches leaves of many coarser levels."""
    segs = []
    g = 8
    for i in range(g):
        for j in range(g):
            cx, cy = -r0 / 2 + (i + 0.5) * r0 / g, -r0 / 2 + (j + 0.5) * r0 / g
            h = 0.2 * r0 / g
            segs.append(((cx - h, cy), (cx + h, cy), 1))
    for k in range(n_shell):
        d = 2 * r0 * 2 ** k
        for q in range(per):
            a = 2 * math.pi * q / per + 0.3 + 0.1 * k
            cx, cy = d * math.cos(a), d * math.sin(a)
            tx, ty = -math.sin(a), math.cos(a)
            h = d / 16
            segs.append(((cx - h * tx, cy - h * ty), (cx + h * tx, cy + h * ty), 2))
    return inputs.assemble(segs)


def lone_crack_and_swarm():
    """A swarm of 25 small cracks near the origin and one 4 m crack 100 m
    away: with leaf_size 16 the lone crack's quadrant is a leaf of level 1."""
    segs = inputs.random_fracture_segments(25, 6.0, 0.4, 1.5, 8, seed=41)
    segs.append(((98.0, 100.0), (102.0, 100.0), 10))
    return inputs.assemble(segs)


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=8, adaptive=True)


@pytest.mark.parametrize("win", [(0.0, 10.0), (0.0, 1e-4), (30.0, 90.0)])
def test_adaptive_matvec_matches_oracle(ctx, win):
    xy = small_clustered()
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    info = tree.info()
    assert info["adaptive"] == 1 and info["depth"] >= 4 and info["leaf_level_min"] <= 3, info
    x = inputs.unknowns(N, seed=51)
    y = ctx.matvec(tree, dev(x), win[0], win[1]).cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, win[0], win[1])
    e = block_rel_err(y, ref, N)
    print(f"window {win}: adaptive FMM vs oracle {e:.2e}, {info}")
    assert e < FMM_TOL
    ctx.device_check()


def test_leaf_above_level_two():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16, adaptive=True)
    xy = lone_crack_and_swarm()
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    info = tree.info()
    assert info["leaf_level_min"] == 1 and info["depth"] >= 4, info
    x = inputs.unknowns(N, seed=52)
    y = ctx.matvec(tree, dev(x), 0.0, 10.0).cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, 0.0, 10.0)
    assert block_rel_err(y, ref, N) < FMM_TOL
    ctx.device_check()


@pytest.mark.parametrize("mode", ["fmm", "fmm+precise"])
def test_many_records_per_leaf(ctx, mode):
    xy = graded()
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    info = tree.info()
    print(info)
    assert info["max_leaf_records"] > 32 and info["depth"] >= 10, info
    x = inputs.unknowns(N, seed=53)
    y = ctx.matvec(tree, dev(x), 0.0, 10.0, mode=mode).cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, 0.0, 10.0)
    assert block_rel_err(y, ref, N) < FMM_TOL
    ctx.device_check()


def test_adaptive_gmres_matches_oracle(ctx):
    xy = small_clustered()
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    loads = dict(sigma_H=20e6, sigma_h=10e6, p_f=25e6, p0=0.0)
    b = ctx.rhs(tree, system="pressure", **loads)
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-8, mode="fmm")
    assert info["converged"]
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), oracle.rhs(xy, system="pressure", **loads), N)
    assert block_rel_err(x.cpu().numpy(), ref, N) < 1e-3
    ctx.device_check()


@pytest.fixture(scope="module")
def clustered10k():
    xy, _ = inputs.clustered_fractures()
    return xy


@pytest.mark.parametrize("n, tol", [(8, FMM_TOL), (12, 2e-5)])
def test_clustered_10k_against_dense(clustered10k, n, tol):
    xy = clustered10k
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=n, leaf_size=32, adaptive=True)
    ta = ctx.build_tree(dev(xy))
    ia = ta.info()
    tu = ctx.build_tree(dev(xy), adaptive=False)          # uniform, automatic depth
    iu = tu.info()
    print("adaptive", ia, "\nuniform", iu)
    # the longest (sparse) cracks cap the uniform depth everywhere; the
    # adaptive tree refines the swarms past that cap
    assert ia["leaf_level_min"] < ia["depth"] and ia["depth"] > iu["depth"]
    assert ia["n_p2p_pairs"] < iu["n_p2p_pairs"]
    x = dev(inputs.unknowns(N, seed=54))
    yd = ctx.matvec(ta, x, 0.0, 10.0, mode="dense").cpu().numpy()
    ya = ctx.matvec(ta, x, 0.0, 10.0).cpu().numpy()
    yu = ctx.matvec(tu, x, 0.0, 10.0).cpu().numpy()
    ea, eu = block_rel_err(ya, yd, N), block_rel_err(yu, yd, N)
    print(f"n = {n}: adaptive vs dense {ea:.2e}, uniform vs dense {eu:.2e}")
    assert ea < tol and eu < tol
    ctx.device_check()


def test_batched_adaptive_equals_alone(ctx):
    geos = [small_clustered(), graded(), lone_crack_and_swarm(), inputs.single_crack(64, 0.5)]
    trees = [ctx.build_tree(dev(g)) for g in geos]
    xs = [inputs.unknowns(g.shape[1], seed=60 + i) for i, g in enumerate(geos)]
    batch = ctx.batch(trees)
    y = batch.matvec(dev(np.concatenate(xs)), 10.0).cpu().numpy()
    for i, (t, g) in enumerate(zip(trees, geos)):
        n = g.shape[1]
        alone = ctx.matvec(t, dev(xs[i]), 0.0, 10.0).cpu().numpy()
        assert block_rel_err(y[batch.offsets[i]:batch.offsets[i + 1]], alone, n) < 1e-5
    ctx.device_check()


def test_autotune_chooses_tree_kind(clustered10k):
    """The tuner tries both tree kinds; its choice on the clustered set meets
    the bound against the dense product, and a tree built with it (kind
    included) reproduces the tuner's error."""
    xy = clustered10k
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)
    x = dev(inputs.unknowns(N, seed=55))
    best = ctx.autotune(dev(xy), x, 10.0, orders=[8], leaves=[16, 32], max_rel_err=1e-5)
    print("autotune on the clustered set:", best)
    assert best["err"] <= 1e-5 and best["adaptive"] in (False, True)
    t = ctx.build_tree(dev(xy), n_cheb=best["n_cheb"], leaf_size=best["leaf_size"], adaptive=best["adaptive"])
    assert t.info()["adaptive"] == int(best["adaptive"])
    yd = ctx.matvec(t, x, 0.0, 10.0, mode="dense").cpu().numpy()
    y = ctx.matvec(t, x, 0.0, 10.0).cpu().numpy()
    assert block_rel_err(y, yd, N) < 1e-5
    ctx.device_check()


def model_cost(info, n=8):
    """The library's cost model of one product (near pairs, interaction pairs
    scaled by (n/8)^4, cells), restated."""
    return 21.5e-12 * info["n_p2p_pairs"] + 3.5e-9 * (n / 8) ** 4 * info["n_m2l_pairs"] + 25e-9 * info["n_cells"]


def test_auto_tree_kind(clustered10k):
    """adaptive = "auto" builds both trees and keeps the one with the lower
    model cost: the adaptive tree on the clustered set; on an evenly spread
    random set, whichever the model prefers.  The kept tree is that kind's
    tree (same counts), and its product matches the dense one."""
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=32, adaptive="auto")
    rand, _ = inputs.random_fractures(n_frac=60, box=110.0, elems=100, seed=77)
    for name, xy in (("clustered", clustered10k), ("random", rand)):
        N = xy.shape[1]
        t = ctx.build_tree(dev(xy))
        ia = t.info()
        iu = ctx.build_tree(dev(xy), adaptive=False).info()
        ic = ctx.build_tree(dev(xy), adaptive=True).info()
        want = 1 if model_cost(ic) < model_cost(iu) else 0
        print(name, "kept", ia["adaptive"], "model uniform", model_cost(iu), "adaptive", model_cost(ic))
        assert ia["adaptive"] == want
        kept = ic if want else iu
        assert (ia["n_cells"], ia["n_p2p_pairs"], ia["n_m2l_pairs"]) == \
            (kept["n_cells"], kept["n_p2p_pairs"], kept["n_m2l_pairs"])
        if name == "clustered":
            assert want == 1
        x = dev(inputs.unknowns(N, seed=56))
        yd = ctx.matvec(t, x, 0.0, 10.0, mode="dense").cpu().numpy()
        y = ctx.matvec(t, x, 0.0, 10.0).cpu().numpy()
        assert block_rel_err(y, yd, N) < FMM_TOL
    ctx.device_check()

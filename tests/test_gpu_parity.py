"""GPU path (C ABI through the Python binding) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances: the pair kernels run in FP32 with FP64 accumulation of the
result; a product row sums O(N) terms of mixed sign, so the expected
relative error (max-norm per output block) is ~1e-6..1e-5 for the dense
path.  The FMM adds its Chebyshev truncation error (n = 8 nodes per
dimension) which stays below 1e-4 here; the solution parity bar is 1e-3."""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev, small_random_set

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
MATVEC_TOL = {"dense": 2e-5, "fmm": 2e-4}


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)


@pytest.fixture(scope="module")
def crack():
    return inputs.single_crack(200, 1.0)


@pytest.fixture(scope="module")
def rset():
    return small_random_set()


@pytest.mark.parametrize("mode", ["dense", "fmm"])
@pytest.mark.parametrize("win", [(0.0, 10.0), (0.0, 1e-4), (0.0, 1e6), (5.0, 20.0)])
def test_matvec_single_crack(ctx, crack, mode, win):
    N = crack.shape[1]
    tree = ctx.build_tree(dev(crack))
    x = inputs.unknowns(N, seed=11)
    y = ctx.matvec(tree, dev(x), win[0], win[1], mode=mode).cpu().numpy()
    ref = oracle.matvec(MAT, crack, x, win[0], win[1])
    assert block_rel_err(y, ref, N) < MATVEC_TOL[mode]


@pytest.mark.parametrize("mode", ["dense", "fmm"])
@pytest.mark.parametrize("win", [(0.0, 10.0), (30.0, 90.0)])
def test_matvec_random_fractures(ctx, rset, mode, win):
    xy, _ = rset
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    if mode == "fmm":
        assert tree.info()["depth"] >= 2          # the far field is exercised
    x = inputs.unknowns(N, seed=12)
    y = ctx.matvec(tree, dev(x), win[0], win[1], mode=mode).cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, win[0], win[1])
    assert block_rel_err(y, ref, N) < MATVEC_TOL[mode]


@pytest.mark.parametrize("mode", ["dense", "fmm"])
def test_history_apply(ctx, rset, mode):
    xy, _ = rset
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    times = [0.0, 10.0, 25.0, 40.0, 70.0]          # H = 3 past steps, observation at 70 s
    hist = np.stack([inputs.unknowns(N, seed=20 + k) for k in range(3)])
    rhs0 = inputs.unknowns(N, seed=30) * 1e9
    got = ctx.history_apply(tree, dev(hist), times, dev(rhs0), mode=mode).cpu().numpy()
    ref = rhs0 - oracle.history(MAT, xy, hist, times)
    corr_got, corr_ref = rhs0 - got, rhs0 - ref
    assert block_rel_err(corr_got, corr_ref, N) < MATVEC_TOL[mode]


@pytest.mark.parametrize("system", ["pressure", "impermeable", "rate"])
@pytest.mark.parametrize("mode", ["dense", "fmm"])
def test_gmres_matches_direct_solve(ctx, crack, system, mode):
    N = crack.shape[1]
    tree = ctx.build_tree(dev(crack))
    dt = 10.0
    # RATE rows carry only the far field and p0 (the injection is a given Dq):
    # give it in-situ stresses so that the system is not trivial
    loads = dict(sigma_H=3e6, sigma_h=2e6, p_f=1e6, p0=5e5) if system == "rate" else dict(p_f=1e6)
    b = ctx.rhs(tree, **{"sigma_H": 0.0, "sigma_h": 0.0, "p0": 0.0, **loads}, system=system)
    b_ref = oracle.rhs(crack, **loads, system=system)
    assert np.allclose(b.cpu().numpy(), b_ref, rtol=1e-14, atol=1e-6)
    x, info = ctx.gmres_solve(tree, dt, b, system=system, tol=1e-5, mode=mode)
    assert info["converged"]
    ref = oracle.solve(oracle.assemble(MAT, crack, dt), b_ref, N, system)
    nb = 3 if system == "pressure" else 2
    assert block_rel_err(x.cpu().numpy(), ref, N, nb) < 1e-3


def test_tree_partitions_elements(ctx, rset):
    xy, _ = rset
    tree = ctx.build_tree(dev(xy))
    info = tree.info()
    assert info["n_elements"] == xy.shape[1]
    assert info["n_leaves"] >= 1 and info["n_cells"] >= info["n_leaves"]
    assert info["n_p2p_pairs"] >= xy.shape[1]

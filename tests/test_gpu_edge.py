"""Edge cases of the GPU path against the FP64 oracle: one element, two
elements, a set smaller than one leaf (no far field), a nearly empty time
window, and inputs the boundary must reject without leaving the context
unusable."""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import DDM_EINVAL, Context, DDMError

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
# With so few elements a row can be a near cancellation of the FP64
# own-element term and the FP32 adjacent-element term (two elements, window
# (5, 20) s: +112 and -152).  The adjacent term stays accurate because
# the close-pair dislocation field takes the window difference in closed
# form where both sides are at large u (no cancellation of the two sides'
# undrained - drained constant).
TOL = {"dense": 2e-5, "fmm": 2e-4}


@pytest.fixture(scope="module")
def ctx():
    return Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)


@pytest.mark.parametrize("n", [1, 2, 10])
@pytest.mark.parametrize("mode", ["dense", "fmm"])
@pytest.mark.parametrize("win", [(0.0, 10.0), (5.0, 20.0)])
def test_few_elements_match_oracle(ctx, n, mode, win):
    """1 element (own-element block only), 2 elements, and 10 < leaf size
    (depth 0: every pair is near)."""
    xy = inputs.single_crack(n, 1.0)
    tree = ctx.build_tree(dev(xy))
    if n < 32:
        assert tree.info()["n_m2l_pairs"] == 0
    x = inputs.unknowns(n, seed=5 + n)
    y = ctx.matvec(tree, dev(x), win[0], win[1], mode=mode).cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, win[0], win[1])
    assert block_rel_err(y, ref, n) < TOL[mode]
    tree.close()
    ctx.device_check()


def test_single_element_solve_matches_direct(ctx):
    xy = inputs.single_crack(1, 0.5)
    tree = ctx.build_tree(dev(xy))
    b = ctx.rhs(tree, p_f=1e6, system="pressure")
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-10, mode="fmm")
    assert info["converged"]
    b_ref = oracle.rhs(xy, p_f=1e6, system="pressure")
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), b_ref, 1, "pressure")
    assert block_rel_err(x.cpu().numpy(), ref, 1) < 1e-6
    tree.close()


@pytest.mark.parametrize("win", [(7.0, 7.0), (5.0, 3.0), (-1.0, 2.0)])
def test_invalid_window_rejected(ctx, win):
    """The window must satisfy 0 <= tau_lo < tau_hi."""
    xy = inputs.single_crack(20, 1.0)
    tree = ctx.build_tree(dev(xy))
    x = dev(inputs.unknowns(20, seed=3))
    for mode in ("dense", "fmm"):
        with pytest.raises(DDMError) as e:
            ctx.matvec(tree, x, win[0], win[1], mode=mode)
        assert e.value.status == DDM_EINVAL
    tree.close()
    ctx.device_check()


def test_nearly_empty_window_is_small(ctx):
    """K(tau + eps) - K(tau) -> 0: a window of 1e-9 s at tau = 7 s."""
    xy = inputs.single_crack(200, 1.0)
    tree = ctx.build_tree(dev(xy))
    x = dev(inputs.unknowns(200, seed=3))
    full = ctx.matvec(tree, x, 0.0, 10.0, mode="fmm").abs().max().item()
    for mode in ("dense", "fmm"):
        y = ctx.matvec(tree, x, 7.0, 7.0 + 1e-9, mode=mode)
        assert y.abs().max().item() <= 1e-5 * full
    tree.close()


def _bad_geometry(kind):
    if kind == "empty":
        return torch.empty(0, dtype=torch.float64, device="cuda")
    xy = inputs.single_crack(8, 1.0).copy()
    if kind == "zero_length":
        xy[2, 3], xy[3, 3] = xy[0, 3], xy[1, 3]      # element 3: both end points equal
    else:
        xy[0, 5] = np.nan
    return dev(xy)


@pytest.mark.parametrize("kind", ["empty", "zero_length", "nan"])
def test_bad_geometry_rejected_context_stays_usable(ctx, kind):
    with pytest.raises(DDMError) as e:
        ctx.build_tree(_bad_geometry(kind))
    assert e.value.status == DDM_EINVAL
    # the context still works
    xy = inputs.single_crack(40, 1.0)
    tree = ctx.build_tree(dev(xy))
    x = inputs.unknowns(40, seed=9)
    y = ctx.matvec(tree, dev(x), 0.0, 10.0, mode="fmm").cpu().numpy()
    assert block_rel_err(y, oracle.matvec(MAT, xy, x, 0.0, 10.0), 40) < TOL["fmm"]
    tree.close()
    ctx.device_check()


@pytest.mark.parametrize("geom", ["crack", "random"])
@pytest.mark.parametrize("win", [(0.0, 10.0), (5.0, 20.0)])
def test_exact_dense_matches_oracle_tightly(ctx, geom, win):
    """DDM_MODE_DENSE | DDM_MODE_PRECISE: FP64 geometry, dislocation pairs
    (the exact element integral) at every distance and an 8-point FP64
    Gauss rule for the fluid source, i.e. the oracle's product up to its
    quadrature tolerance; the FP32 paths are held to 2e-5 / 2e-4."""
    from gpu_common import small_random_set
    xy = inputs.single_crack(200, 1.0) if geom == "crack" else small_random_set()[0]
    n = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    x = inputs.unknowns(n, seed=21)
    y = ctx.matvec(tree, dev(x), win[0], win[1], mode="dense+precise").cpu().numpy()
    ref = oracle.matvec(MAT, xy, x, win[0], win[1])
    assert block_rel_err(y, ref, n) < 1e-7
    tree.close()


def test_grid_barrier_timeout_reported_and_context_recovers(ctx):
    """A poll limit of one makes the grid barriers of the GMRES
    orthogonalisation give up (no kernel is broken: the waits return early
    and raise the context's error word).  The solve reports DDM_ETIMEOUT,
    resets the barrier and the word, and the next solve on the same context,
    at the default limit, converges to the oracle's direct solution."""
    from paper_1812_05087_gb300.ddm import DDM_ETIMEOUT
    xy = inputs.single_crack(64, 1.0)
    N = xy.shape[1]
    tree = ctx.build_tree(dev(xy))
    b = ctx.rhs(tree, p_f=1e6, system="impermeable")
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(DDMError) as e:
            ctx.gmres_solve(tree, 10.0, b, system="impermeable", tol=1e-8)
        assert e.value.status == DDM_ETIMEOUT
    finally:
        ctx.set_wait_limit(0)
    ctx.device_check()                     # the word was cleared by the solve
    x, info = ctx.gmres_solve(tree, 10.0, b, system="impermeable", tol=1e-8)
    assert info["converged"]
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), oracle.rhs(xy, p_f=1e6, system="impermeable"), N,
                       "impermeable")
    assert block_rel_err(x.cpu().numpy(), ref, N, blocks=2) < 1e-4
    ctx.device_check()
    tree.close()

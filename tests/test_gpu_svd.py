"""Compressed M2L operators (the SVD compression of black-box FMM operators
that paper Sec. 3 cites; ddm_set_m2l_compression).

- Mode 1 at every order with a rank (n = 8 ... 16), on forced depth 4 and on
  the automatic depth, for the step window and a history window: the
  compressed FMM product against the dense product on the same tree, and
  against the uncompressed FMM product.  The compression adds the
  truncation error of the rank-k bases to the interpolation error; the bar
  is 3e-5.
- A GMRES solve whose operator takes the compressed M2L, against the
  oracle's direct solution.
- The automatic mode: orders below 10 never compress; at n = 12 a window
  compresses after 128 products (the M2L stage then runs as three grouped
  launches instead of one), and the product stays within the bar.
- An unknown mode is rejected."""
import numpy as np
import pytest

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context, DDMError

from gpu_common import block_rel_err, dev, small_random_set

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
TOLC = 3e-5


@pytest.fixture(scope="module")
def mid_set():
    segs = inputs.random_fracture_segments(40, 60.0, 2.0, 8.0, 40, 5)
    return inputs.assemble(segs)


def m2l_launches(ctx, tree, x, lo, hi):
    """M2L launches of one product (the launch counters run whether or not
    profiling is on; a read returns and clears them)."""
    ctx.profile_read()
    ctx.profile(True)
    ctx.matvec(tree, x, lo, hi, mode="fmm")
    st = ctx.profile_read()
    ctx.profile(False)
    return st["m2l"][1]


@pytest.mark.parametrize("n", [8, 10, 12, 14, 16])
@pytest.mark.parametrize("depth", [4, 0])
def test_compressed_product_every_order(mid_set, n, depth):
    xy = mid_set
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=n, leaf_size=1 if depth else 16, max_depth=depth)
    tree = ctx.build_tree(dev(xy))
    if depth:
        assert tree.info()["depth"] == depth
    x = dev(inputs.unknowns(N, seed=51))
    for lo, hi in ((0.0, 10.0), (20.0, 50.0)):
        ctx.set_m2l_compression(0)
        yf = ctx.matvec(tree, x, lo, hi, mode="fmm").cpu().numpy()
        ctx.set_m2l_compression(1)
        yc = ctx.matvec(tree, x, lo, hi, mode="fmm").cpu().numpy()
        assert m2l_launches(ctx, tree, x, lo, hi) == 3
        ref = ctx.matvec(tree, x, lo, hi, mode="dense").cpu().numpy()
        e_c, e_f, e_cf = block_rel_err(yc, ref, N), block_rel_err(yf, ref, N), block_rel_err(yc, yf, N)
        print(f"n={n} depth={tree.info()['depth']} window=({lo},{hi}) compressed {e_c:.2e} full {e_f:.2e} "
              f"compressed-vs-full {e_cf:.2e}")
        assert e_c < TOLC and e_cf < TOLC
    ctx.device_check()


def test_compressed_solve_matches_oracle():
    xy, segs = small_random_set(n_frac=16, box=24.0, elems=40, seed=9)
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=12, leaf_size=8)
    ctx.set_m2l_compression(1)
    tree = ctx.build_tree(dev(xy))
    assert tree.info()["depth"] >= 2
    loads = dict(sigma_H=30e6, sigma_h=25e6, p_f=10e6, p0=0.0)
    b = ctx.rhs(tree, system="pressure", **loads)
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-6, mode="fmm")
    assert info["converged"]
    assert m2l_launches(ctx, tree, x, 0.0, 10.0) == 3
    ref = oracle.solve(oracle.assemble(MAT, xy, 10.0), oracle.rhs(xy, system="pressure", **loads), N)
    assert block_rel_err(x.cpu().numpy(), ref, N) < 1e-3
    ctx.device_check()


def test_automatic_mode(mid_set):
    xy = mid_set
    N = xy.shape[1]
    x = dev(inputs.unknowns(N, seed=52))
    # n = 8: never compressed
    c8 = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    t8 = c8.build_tree(dev(xy))
    y = c8.matvec(t8, x, 0.0, 10.0, mode="fmm")
    for _ in range(140):
        c8.matvec(t8, x, 0.0, 10.0, mode="fmm", out=y)
    assert m2l_launches(c8, t8, x, 0.0, 10.0) == 1
    # n = 12: full operators for the first 128 products, compressed after
    c12 = Context(inputs.MATERIAL, n_cheb=12, leaf_size=16)
    t12 = c12.build_tree(dev(xy))
    y = c12.matvec(t12, x, 0.0, 10.0, mode="fmm")
    for _ in range(100):
        c12.matvec(t12, x, 0.0, 10.0, mode="fmm", out=y)
    assert m2l_launches(c12, t12, x, 0.0, 10.0) == 1
    for _ in range(40):
        c12.matvec(t12, x, 0.0, 10.0, mode="fmm", out=y)
    assert m2l_launches(c12, t12, x, 0.0, 10.0) == 3
    ref = c12.matvec(t12, x, 0.0, 10.0, mode="dense").cpu().numpy()
    assert block_rel_err(y.cpu().numpy(), ref, N) < TOLC
    # another window starts its own count
    assert m2l_launches(c12, t12, x, 20.0, 50.0) == 1
    c12.device_check()


def test_bad_mode_rejected():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    with pytest.raises(DDMError):
        ctx.set_m2l_compression(3)
    with pytest.raises(DDMError):
        ctx.set_m2l_compression(-1)
    with pytest.raises(DDMError):
        ctx.set_m2l_compression(1, rank=12)
    with pytest.raises(DDMError):
        ctx.set_m2l_compression(1, rank=520)


def test_rank_override_and_change(mid_set):
    """A lower rank stays within the bar at n = 12; changing the rank on a
    tree drops its cached sets and builds new ones of the new rank."""
    xy = mid_set
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=12, leaf_size=16)
    tree = ctx.build_tree(dev(xy))
    x = dev(inputs.unknowns(N, seed=53))
    ref = ctx.matvec(tree, x, 0.0, 10.0, mode="dense").cpu().numpy()
    for rank in (64, 128, 48, 0):
        ctx.set_m2l_compression(1, rank=rank)
        y = ctx.matvec(tree, x, 0.0, 10.0, mode="fmm").cpu().numpy()
        assert m2l_launches(ctx, tree, x, 0.0, 10.0) == 3
        e = block_rel_err(y, ref, N)
        print(f"rank={rank} err={e:.2e}")
        assert e < TOLC
    ctx.device_check()

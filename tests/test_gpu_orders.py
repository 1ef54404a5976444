"""FMM product at every supported Chebyshev order and at forced tree depths,
against the dense product on the same tree (the dense product is itself held
to the FP64 oracle by the parity tests).  This covers the tensor-core M2L
with ragged K chunks and partial 128-row slices (4n^2 = 16 ... 1024), the
fused upward pass (P2M + M2M through several levels, including depth 2 where
no M2M runs) and the fused L2L chains.

Expected FMM error: the Chebyshev interpolation error of the far field,
falling roughly geometrically with n down to the FP32 floor (~7e-7 of the
block maximum); the bars are about 10x the values measured on GB300 with
the automatic depth (n = 2: 1.7e-4, n = 4: 1.7e-5, n = 6: 2.7e-6,
n >= 8: 6.7e-7)."""
import numpy as np
import pytest

from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
TOL = {2: 2e-3, 4: 2e-4, 6: 3e-5, 8: 1e-5, 10: 1e-5, 12: 1e-5, 14: 1e-5, 16: 1e-5}


@pytest.fixture(scope="module")
def mid_set():
    segs = inputs.random_fracture_segments(40, 60.0, 2.0, 8.0, 40, 5)
    return inputs.assemble(segs)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14, 16])
def test_fmm_every_order(mid_set, n):
    xy = mid_set
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=n, leaf_size=1, max_depth=4)
    tree = ctx.build_tree(dev(xy))
    assert tree.info()["depth"] == 4
    x = dev(inputs.unknowns(N, seed=41))
    for lo, hi in ((0.0, 10.0), (20.0, 50.0)):
        y = ctx.matvec(tree, x, lo, hi, mode="fmm").cpu().numpy()
        ref = ctx.matvec(tree, x, lo, hi, mode="dense").cpu().numpy()
        err = block_rel_err(y, ref, N)
        print(f"n={n} window=({lo},{hi}) err={err:.2e}")
        assert err < TOL[n]
    ctx.device_check()


@pytest.mark.parametrize("depth", [1, 2, 3, 4, 5, 6])
def test_fmm_forced_depth(mid_set, depth):
    xy = mid_set
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=1, max_depth=depth)
    tree = ctx.build_tree(dev(xy))
    assert tree.info()["depth"] == depth
    x = dev(inputs.unknowns(N, seed=42))
    y = ctx.matvec(tree, x, 0.0, 10.0, mode="fmm").cpu().numpy()
    ref = ctx.matvec(tree, x, 0.0, 10.0, mode="dense").cpu().numpy()
    err = block_rel_err(y, ref, N)
    print(f"depth={depth} err={err:.2e}")
    assert err < 1e-5
    # a second product on the same tree (internal cells zeroed again)
    y2 = ctx.matvec(tree, x, 0.0, 10.0, mode="fmm").cpu().numpy()
    assert block_rel_err(y2, ref, N) < 1e-5
    ctx.device_check()


def test_overlapped_product_equals_serial(mid_set):
    """The default product runs the near field concurrently with the far field
    (two streams); with stage profiling on it runs serially.  Both schedules
    compute the same sums (up to the order of the M2L atomics)."""
    xy = mid_set
    N = xy.shape[1]
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    tree = ctx.build_tree(dev(xy))
    assert tree.info()["depth"] >= 3
    x = dev(inputs.unknowns(N, seed=43))
    for lo, hi in ((0.0, 10.0), (20.0, 50.0)):
        y_par = ctx.matvec(tree, x, lo, hi, mode="fmm").cpu().numpy()
        ctx.profile(True)
        y_ser = ctx.matvec(tree, x, lo, hi, mode="fmm").cpu().numpy()
        ctx.profile(False)
        ctx.profile_read()
        assert block_rel_err(y_par, y_ser, N) < 1e-6
    ctx.device_check()

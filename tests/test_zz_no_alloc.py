"""The allocation-free dense product (ddm_matvec_dense_static).

Some callers cannot allocate device memory where they need a product (a
real-time loop that forbids allocation after start-up, or code inside
another framework's fixed memory budget).  For them the library offers one
entry point whose only scratch is a fixed device array inside the library.
This test calls it through the C ABI twice in a row, on different inputs,
and checks each result against the regular dense product at the tolerance
the dense parity tests use, and once directly against the FP64 oracle;
sizes beyond the array's capacity and overlapping vectors are rejected
before any GPU work, and invalid geometry gives NaN outputs without
spoiling the next call.  It lives in its own file so that it runs last."""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05087_gb300.ddm as ddm
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context

from gpu_common import block_rel_err, dev, small_random_set

DENSE_TOL = 2e-5


@pytest.mark.gpu
def test_static_dense_matches_dense_on_two_calls():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)
    xy, _ = small_random_set()
    N = xy.shape[1]
    d_xy = dev(xy)
    tree = ctx.build_tree(d_xy)
    y = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    for seed, win in ((31, (0.0, 10.0)), (32, (5.0, 20.0))):
        x = dev(inputs.unknowns(N, seed=seed))
        ref = ctx.matvec(tree, x, win[0], win[1], mode="dense").cpu().numpy()
        ddm.ddm_matvec_dense_static(ctx.ptr, d_xy, win[0], win[1], x, y)
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert block_rel_err(got, ref, N) < DENSE_TOL


@pytest.mark.gpu
def test_static_dense_rejects_oversize():
    ctx = Context(inputs.MATERIAL)
    n = ddm.STATIC_MAX_ELEMENTS + 1
    xy = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    x = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    y = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_matvec_dense_static(ctx.ptr, xy, 0.0, 10.0, x, y)
    assert e.value.status == ddm.DDM_EINVAL


@pytest.mark.gpu
def test_static_dense_matches_oracle():
    ctx = Context(inputs.MATERIAL)
    xy = inputs.single_crack(40, 1.0)
    N = xy.shape[1]
    x = inputs.unknowns(N, seed=33)
    y = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    ddm.ddm_matvec_dense_static(ctx.ptr, dev(xy), 0.0, 10.0, dev(x), y)
    ref = oracle.matvec(inputs.material_tuple(), xy, x, 0.0, 10.0)
    assert block_rel_err(y.cpu().numpy(), ref, N) < DENSE_TOL


@pytest.mark.gpu
def test_static_dense_invalid_geometry_and_overlap():
    ctx = Context(inputs.MATERIAL)
    xy = inputs.single_crack(16, 1.0)
    N = xy.shape[1]
    x = dev(inputs.unknowns(N, seed=34))
    y = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    bad = xy.copy()
    bad[2, 5], bad[3, 5] = bad[0, 5], bad[1, 5]          # element 5 has zero length
    ddm.ddm_matvec_dense_static(ctx.ptr, dev(bad), 0.0, 10.0, x, y)
    assert torch.isnan(y).all()
    ddm.ddm_matvec_dense_static(ctx.ptr, dev(xy), 0.0, 10.0, x, y)    # the flag is cleared per call
    ref = ctx.matvec(ctx.build_tree(dev(xy)), x, 0.0, 10.0, mode="dense").cpu().numpy()
    assert block_rel_err(y.cpu().numpy(), ref, N) < DENSE_TOL
    buf = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    buf[:3 * N] = x
    with pytest.raises(ddm.DDMError) as e:       # y starts inside x's 3N range
        ddm.ddm_matvec_dense_static(ctx.ptr, dev(xy), 0.0, 10.0, buf[:3 * N], buf[N:])
    assert e.value.status == ddm.DDM_EINVAL

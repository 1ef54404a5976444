"""Helpers shared by the GPU parity tests (inputs and error metrics only)."""
import numpy as np
import torch

from paper_1812_05087_gb300 import inputs


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def block_rel_err(got, ref, n, blocks=3, floor=1e-4):
    """max over component blocks of ||got - ref||_inf / ||ref||_inf.  A block
    whose largest entry is below `floor` times the largest entry of all blocks
    is zero at the solver tolerances used here (a 1e-5 relative residual
    leaves solution noise near 1e-4 of the largest block; e.g. the shear
    block of a pressurised straight crack is exactly zero in the oracle and
    ~1e-12 against an opening of ~3e-4 on the GPU); it is measured against
    that floor instead."""
    got, ref = np.asarray(got), np.asarray(ref)
    top = np.max(np.abs(ref[:blocks * n]))
    errs = []
    for b in range(blocks):
        r = ref[b * n:(b + 1) * n]
        g = got[b * n:(b + 1) * n]
        scale = max(np.max(np.abs(r)), floor * top)
        if scale == 0:
            continue
        errs.append(np.max(np.abs(g - r)) / scale)
    return max(errs)


def small_random_set(n_frac=12, box=20.0, elems=30, seed=7):
    segs = inputs.random_fracture_segments(n_frac, box, 2.0, 6.0, elems, seed)
    return inputs.assemble(segs), segs

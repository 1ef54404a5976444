"""Continuous-batching server: requests that arrive while others are being
solved join later rounds; every request's result in the mix equals the same
request served alone (and, for a small multi-step case, the FP64 oracle's
time marching)."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1812_05087_gb300 import inputs
from paper_1812_05087_gb300.ddm import Context, Server

from gpu_common import block_rel_err, dev

pytestmark = pytest.mark.gpu
MAT = inputs.material_tuple()
LOADS = dict(sigma_H=3e6, sigma_h=2e6, p_f=5e6, p0=0.0)


def requests():
    out = [(inputs.single_crack(48, 0.5), 3)]
    for k, (nf, el, box, steps) in enumerate([(3, 20, 8.0, 1), (6, 25, 12.0, 2), (10, 30, 20.0, 1),
                                             (2, 60, 6.0, 4)]):
        segs = inputs.random_fracture_segments(nf, box, 1.0, min(5.0, box / 2), el, seed=200 + k)
        out.append((inputs.assemble(segs), steps))
    return out


def wait(srv, tickets, limit=180.0):
    t0 = time.time()
    res = {}
    while len(res) < len(tickets):
        assert time.time() - t0 < limit, "server did not finish in time"
        for t in tickets:
            if t in res:
                continue
            r = srv.poll(t)
            if r["poll"] != 6:           # DDM_PENDING
                res[t] = r
        time.sleep(0.005)
    return res


def test_mix_equals_alone_and_oracle():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    reqs = requests()
    dt = 10.0
    # mix: two requests first, the rest while the first are running
    srv = Server(ctx, max_active=8, tol=1e-5)
    xys = [dev(g) for g, _ in reqs]
    outs = [torch.zeros(3 * g.shape[1], dtype=torch.float64, device="cuda") for g, _ in reqs]
    tickets = [srv.submit(xys[i], outs[i], dt, reqs[i][1], **LOADS) for i in range(2)]
    time.sleep(0.05)
    tickets += [srv.submit(xys[i], outs[i], dt, reqs[i][1], **LOADS) for i in range(2, len(reqs))]
    res = wait(srv, tickets)
    srv.close()
    for t in tickets:
        assert res[t]["status"] == 0 and res[t]["latency_ms"] > 0
    mix = [o.cpu().numpy() for o in outs]
    # alone: each request in a fresh server of its own
    for i, (g, steps) in enumerate(reqs):
        s1 = Server(ctx, max_active=1, tol=1e-5)
        o = torch.zeros(3 * g.shape[1], dtype=torch.float64, device="cuda")
        t = s1.submit(xys[i], o, dt, steps, **LOADS)
        r = wait(s1, [t])[t]
        s1.close()
        assert r["status"] == 0
        assert block_rel_err(mix[i], o.cpu().numpy(), g.shape[1]) < 2e-4
    # oracle time marching for the single crack (3 steps of 10 s)
    g, steps = reqs[0]
    n = g.shape[1]
    times = [dt * k for k in range(steps + 1)]
    b = oracle.rhs(g, system="pressure", **LOADS)
    ref = oracle.march(MAT, g, times, [b] * steps)[-1]
    assert block_rel_err(mix[0], ref, n) < 1e-3

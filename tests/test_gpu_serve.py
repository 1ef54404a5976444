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


def fracture_set(n_target, seed):
    """A random fracture set of about n_target elements (the serving trace's
    recipe, inputs.serving_geometry)."""
    return inputs.serving_geometry(n_target, seed)


def test_cancel_stops_queued_and_active_requests():
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)
    srv = Server(ctx, max_active=2, tol=1e-5)
    xys = [dev(fracture_set(3000, 700 + k)) for k in range(8)]
    outs = [torch.zeros(3 * (g.numel() // 4), dtype=torch.float64, device="cuda") for g in xys]
    tickets = [srv.submit(g, o, 10.0, 50, **LOADS) for g, o in zip(xys, outs)]
    t0 = time.time()
    while srv.poll(tickets[0])["steps_done"] < 2:
        assert time.time() - t0 < 120.0
        time.sleep(0.01)
    srv.cancel()
    res = wait(srv, tickets, limit=60.0)
    st = [res[t]["status"] for t in tickets]
    assert all(s in (0, 7) for s in st) and st.count(7) >= 6, st
    # the server keeps serving after a cancel
    g = dev(fracture_set(1000, 799))
    o = torch.zeros(3 * (g.numel() // 4), dtype=torch.float64, device="cuda")
    t = srv.submit(g, o, 10.0, 2, **LOADS)
    assert wait(srv, [t])[t]["status"] == 0
    srv.close()


def test_large_request_equals_direct_solve():
    """A request of ~200,000 elements (the top of the serving trace's size
    range) through the server, against the same step solved directly."""
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=32)
    xy = fracture_set(200000, 901)
    N = xy.shape[1]
    assert N > 150000
    g = dev(xy)
    srv = Server(ctx, max_active=4, tol=1e-5)
    o = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t = srv.submit(g, o, 10.0, 1, **LOADS)
    r = wait(srv, [t], limit=300.0)[t]
    srv.close()
    assert r["status"] == 0
    tree = ctx.build_tree(g)
    b = ctx.rhs(tree, system="pressure", **LOADS)
    x, info = ctx.gmres_solve(tree, 10.0, b, system="pressure", tol=1e-5)
    assert info["converged"]
    assert block_rel_err(o.cpu().numpy(), x.cpu().numpy(), N) < 1e-3


def test_server_takes_history_compression_of_its_context():
    """A 40-step request in a server created from a context with the
    time-compressed history sum equals the same march run on that context."""
    ctx = Context(inputs.MATERIAL, n_cheb=8, leaf_size=16)
    ctx.set_history_compression(8, 8, 2.0)
    xy = fracture_set(1500, 950)
    N = xy.shape[1]
    g = dev(xy)
    steps, dt = 40, 10.0
    srv = Server(ctx, max_active=2, tol=1e-6)
    o = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t = srv.submit(g, o, dt, steps, **LOADS)
    r = wait(srv, [t], limit=300.0)[t]
    srv.close()
    assert r["status"] == 0
    tree = ctx.build_tree(g)
    b0 = ctx.rhs(tree, system="pressure", **LOADS)
    hist = torch.zeros(steps, 3 * N, dtype=torch.float64, device="cuda")
    x = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    for h in range(1, steps + 1):
        b = b0.clone()
        if h > 1:
            ctx.history_apply(tree, hist[:h - 1], [dt * k for k in range(h + 1)], b)
        x, info = ctx.gmres_solve(tree, dt, b, x, system="pressure", tol=1e-6)
        hist[h - 1] = x
    assert block_rel_err(o.cpu().numpy(), x.cpu().numpy(), N) < 1e-3

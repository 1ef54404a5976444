"""The N > 1 path of the benchmark on CPU: two gloo ranks on 127.0.0.1.

With N GPUs the product shards only across independent problems (replicas):
each rank builds its own seeded fracture set, times its own products, and
the job's value is all ranks' elements at the slowest rank's time.  These
tests run that host logic (the bench's own helpers) with a real process
group; no GPU and no data-path collective are involved."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        import torch
        import torch.distributed as dist

        import bench
        from paper_1812_05087_gb300 import inputs

        dist.init_process_group("gloo", rank=rank, world_size=world)
        # per-rank timings (ms): product and end-to-end, different on each rank
        mine = [1.0 + rank, 10.0 - 3.0 * rank]
        agreed = bench.max_over_ranks(dist, mine, "cpu")
        seed = bench.replica_seed(rank)
        xy, _ = inputs.random_fractures(seed=seed)
        info = torch.tensor([seed, xy.shape[1]], dtype=torch.int64)
        allinfo = [torch.zeros_like(info) for _ in range(world)]
        dist.all_gather(allinfo, info)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, agreed, [t.tolist() for t in allinfo],
               bench.whole_job_melem_s(world, xy.shape[1], agreed[0]), float(xy[0, 0])))
    except Exception as e:          # reported to the parent, which fails the test
        q.put((rank, "error", repr(e)))


def _run_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(WORLD):
            r = q.get(timeout=180)
            out[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
                p.join()
    return out, [p.exitcode for p in procs]


@pytest.fixture(scope="module")
def ranks():
    return _run_ranks()


def test_ranks_exit_cleanly(ranks):
    out, codes = ranks
    assert sorted(out) == list(range(WORLD))
    for r in out.values():
        assert r[1] != "error", r
    assert codes == [0] * WORLD


def test_timings_are_the_max_over_ranks(ranks):
    out, _ = ranks
    expect = [float(WORLD), 10.0]        # max(1 + rank), max(10 - 3 rank)
    for r in out.values():
        assert r[1] == expect


def test_replicas_are_distinct_problems_of_equal_size(ranks):
    out, _ = ranks
    infos = out[0][2]
    assert infos == out[1][2]            # every rank saw the same gathered table
    seeds = [i[0] for i in infos]
    sizes = [i[1] for i in infos]
    assert len(set(seeds)) == WORLD       # own seeded fracture set per rank
    assert len(set(sizes)) == 1           # same workload size on every rank
    assert out[0][4] != out[1][4]         # and different geometry


def test_whole_job_value_counts_every_rank(ranks):
    out, _ = ranks
    n = out[0][2][0][1]
    slowest_ms = float(WORLD)
    for r in out.values():
        assert r[3] == pytest.approx(WORLD * n / (slowest_ms * 1e-3) / 1e6, rel=1e-15)


def test_reference_arm_runs_on_rank_0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1, WORLD) is None      # other ranks: no work, no line
    assert capsys.readouterr().out == ""

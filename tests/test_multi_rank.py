"""The multi-rank host logic of bench.py on two gloo ranks (CPU, no GPU).

On N GPUs every rank solves its own batch with no data-path collective (replicas of
independent instances and PAQIF systems); the only collectives are the barrier around the
timed steps and the maximum of the step times over ranks.  These tests run that logic with
the gloo backend: the rank/world parsing, the max-over-ranks reduction of every timed figure
(with legs that did not run), the whole-job rate, and that only rank 0 of the reference arm
does work and prints.
"""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        w, r, loc = bench.dist_env()
        # per-rank times (ms) of the legs: A, B, a leg that did not run, the two end-to-end passes
        mine = [1.0 + rank, 10.0 - rank, None, 3.0 * (rank + 1), 0.5]
        got = bench.max_over_ranks(mine, w, torch.device("cpu"))
        rate = bench.job_rate(w, 512, got[1])
        bench_args = argparse.Namespace(ref_systems=1, warmup=0, steps=1)
        ref = bench.run_reference(bench_args) if rank != 0 else "rank 0 not run here"
        dist.barrier()
        q.put((rank, (w, r, loc), got, rate, ref))
    finally:
        dist.destroy_process_group()


def _run():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return {o[0]: o[1:] for o in out}


@pytest.fixture(scope="module")
def ranks():
    return _run()


def test_rank_and_world_from_the_environment(ranks):
    for r in range(WORLD):
        assert ranks[r][0] == (WORLD, r, r)


def test_every_timed_figure_is_the_slowest_ranks(ranks):
    for r in range(WORLD):
        got = ranks[r][1]
        assert got[0] == 2.0  # rank 1's leg A
        assert got[1] == 10.0  # rank 0's leg B
        assert got[2] is None  # a leg that no rank ran
        assert got[3] == 6.0
        assert got[4] == 0.5


def test_whole_job_rate_counts_all_ranks_units(ranks):
    # 2 ranks x 512 solves in the slowest rank's 10 ms
    for r in range(WORLD):
        assert ranks[r][2] == pytest.approx(2 * 512 / 10e-3)


def test_reference_arm_runs_on_rank_0_only(ranks):
    assert ranks[1][3] is None


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks([1.5, None], 1, None) == [1.5, None]
    assert bench.job_rate(1, 512, 100.0) == pytest.approx(5120.0)

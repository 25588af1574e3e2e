"""The multi-GPU form of the benchmark on CPU: two gloo ranks, world_size 2.

Events are independent (Sec. 3 event-level parallelism), so N ranks shard the event stream
with no exchange on the data path; the only collectives are the timing barrier and the
max-over-ranks reduction. These tests run that host logic with the oracle standing in for
the GPU path: the shards must partition the single-process stream exactly, and the job time
must be the slowest rank's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402

WORLD = 2
EVENTS_PER_RANK = 6


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, port: int, cfg_name: str):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(WORLD), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (WORLD, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        cfg = gen.CONFIGS[cfg_name]
        ev = gen.generate(cfg, EVENTS_PER_RANK, first_event=bench.shard_first_event(rank, EVENTS_PER_RANK),
                          with_truth=False)
        p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks)
        res = oracle.run(ev.xy, ev.off, p)
        shards = [None] * WORLD
        dist.all_gather_object(shards, (rank, ev.xy, ev.off, res.npeaks, res.peaks, res.mask, res.nkept,
                                        res.checksum))
        # the job time is the slowest rank's
        assert bench.max_over_ranks(1.0 + 2.5 * rank, dist, "cpu") == 1.0 + 2.5 * (WORLD - 1)
        if rank == 0:
            whole = gen.generate(cfg, WORLD * EVENTS_PER_RANK, with_truth=False)
            ref = oracle.run(whole.xy, whole.off, p)
            shards.sort(key=lambda t: t[0])
            xy = np.concatenate([s[1] for s in shards])
            off = np.concatenate([shards[0][2]] + [s[2][1:] + sum(len(t[1]) for t in shards[:i])
                                                   for i, s in enumerate(shards) if i > 0])
            np.testing.assert_array_equal(xy, whole.xy)
            np.testing.assert_array_equal(off, whole.off)
            np.testing.assert_array_equal(np.concatenate([s[3] for s in shards]), ref.npeaks)
            np.testing.assert_array_equal(np.concatenate([s[4] for s in shards]), ref.peaks)
            np.testing.assert_array_equal(np.concatenate([s[5] for s in shards]), ref.mask)
            np.testing.assert_array_equal(np.concatenate([s[6] for s in shards]), ref.nkept)
            np.testing.assert_array_equal(np.concatenate([s[7] for s in shards]), ref.checksum)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cfg_name", ["plain_small", "plain_paper"])
def test_two_gloo_ranks_partition_the_event_stream(cfg_name):
    mp.spawn(_rank_main, args=(_free_port(), cfg_name), nprocs=WORLD, join=True)


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.shard_first_event(0, 100) == 0 and bench.shard_first_event(3, 100) == 300

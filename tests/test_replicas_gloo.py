"""The N > 1 bench path is replicas only: each rank denoises its own frames,
the job time is the slowest rank's.  The host logic runs here on two CPU
ranks over gloo (no GPU, no data exchanged beyond the timing maximum)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_total_ms = [10.0, 14.0][rank]            # two timed steps on each rank
    slowest = bench.max_over_ranks(local_total_ms, dist, "cpu")
    q.put((rank, bench.replica_seed(bench.SEED, rank), slowest, bench.job_metrics(slowest / 2, world)))
    dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    [p.start() for p in ps]
    res = sorted(q.get(timeout=120) for _ in ps)
    [p.join(timeout=60) for p in ps]
    assert all(p.exitcode == 0 for p in ps)
    seeds = {r[1] for r in res}
    assert len(seeds) == 2                          # distinct frames per replica
    for _, _, slowest, m in res:
        assert slowest == 14.0                       # both ranks agree on the max
        assert m["ms_per_step"] == pytest.approx(7.0)
        assert m["ms_per_frame"] == pytest.approx(3.5)   # 2 frames per 7 ms step
        assert m["fps"] == pytest.approx(2000.0 / 7.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_metrics(2.0, 1) == {"ms_per_step": 2.0, "ms_per_frame": 2.0, "fps": 500.0}

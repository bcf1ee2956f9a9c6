"""The N > 1 benchmark path on CPU with two gloo ranks: each rank draws its own
batch (different seeds, so different inputs), the job time is the slowest
rank's, and the whole-job rate counts every rank's units; the reference arm
runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, port: int, q) -> None:
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    from paper_2512_18345_gb300 import inputs
    seed = inputs.WORKLOADS[bench.WORKLOAD]["seed"]
    g = inputs.rng(bench.rank_seed(seed, rank))
    first = inputs.uniform_residues(g, [65537 * 2 ** 10 + 1], 16)[0].tolist()  # a rank's first input words
    mine = 10.0 + 7.5 * rank                                                     # this rank's time, ms
    slowest = bench.max_over_ranks(mine, 2, "cpu")
    gathered = [None, None]
    dist.all_gather_object(gathered, first)
    q.put((rank, slowest, bench.job_throughput(8 * 400, 2, slowest), gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, gathered in res:
        assert slowest == 17.5                           # max over ranks on every rank
        assert abs(rate - 2 * 8 * 400 / 17.5e-3) < 1e-6  # both ranks' units over the slowest time
        assert gathered[0] != gathered[1]                # the ranks' batches differ


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.rank_seed(7, 0) == 7 and bench.rank_seed(7, 3) == 3007
    assert np.isclose(bench.job_throughput(100, 1, 50.0), 2000.0)
    assert bench.run_reference(None, 2, 1) is None  # the reference arm: ranks other than 0 do no work

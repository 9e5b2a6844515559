"""The multi-GPU benchmark path runs independent replicas (the likelihood is
not sharded across GPUs); its only exchange is the max over ranks of the
timed duration.  Checked here with two gloo ranks on the CPU."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.0, 3.0][rank]
    value, ms_max = bench.aggregate_replicas(ms, units=1000, dist=dist, device="cpu")
    q.put((rank, value, ms_max))
    dist.destroy_process_group()


def test_two_replicas_report_whole_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29511
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, ms_max in res:
        assert ms_max == 3.0
        assert abs(value - 2 * 1000 / 3e-3) < 1e-6

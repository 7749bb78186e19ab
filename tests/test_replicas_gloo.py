"""The multi-GPU arrangement (replicas only) exercised on CPU ranks.

Paths are independent and the loss is a sum over paths, but this build gets
one GPU per job: `bench.py --gpus N` runs N independent replicas (own seed,
own noise, own Theta_0), times each, and reports all ranks' steps over the
slowest rank's time.  Two gloo ranks check the host side of that: distinct
replicas, the max-over-ranks reduction and the job throughput."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import fbsde as F
    seed = bench.replica_seed(7, rank)
    p = F.Problem(kind="bsb", D=3, N=4, M=8, x0=np.array([1.0, 0.5, 1.0]))
    a = F.Arch(kind="fc", width=8, depth=1, act="tanh")
    theta = F.init_params(p, a, seed)
    loss = F.rollout_loss(p, a, theta, seed, 1).loss
    ms = 10.0 + 5.0 * rank  # this rank's timed region (rank 1 is the slower one)
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    losses = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(losses, torch.tensor([loss], dtype=torch.float64))
    dist.barrier()
    if rank == 0:
        out.put((float(t.item()), [float(x.item()) for x in losses],
                 bench.job_throughput(world, 20, float(t.item()))))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    ms_max, losses, value = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert ms_max == 15.0                       # the slowest rank sets the time
    assert losses[0] != losses[1]               # independent replicas (own noise and Theta_0)
    assert value == pytest.approx(2 * 20 / 0.015)  # all ranks' steps / slowest time

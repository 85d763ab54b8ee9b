"""Wavelength sharding over ranks: torch.distributed with the gloo backend, world size 2, on CPU.

Each rank's data path is stood in for by the CPU oracle (this machine has no GPU; the kernels are
covered by the GPU tests). What is checked is the sharding logic of
`paper_1410_0986_gb300.shard`: every wavelength chunk is owned by exactly one rank, the ranks of one
step take distinct chunks, the gradient all-reduce sums the per-rank J^T y contributions into the
full one (J^T y is a sum over wavelengths), and a rank that fails is detected by its peer as an
error instead of a hang.
"""
import datetime
import os
import socket

import numpy as np
import pytest

import workloads
from oracle import born as oborn
from oracle import solve as osolve
from paper_1410_0986_gb300 import shard

N_LAMBDA = 4


def _problem():
    return workloads.small(seed=61, nx=8, ny=7, nz=6, n_src=3, n_det=2, n_lambda=N_LAMBDA)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    return dist


def _gradient_worker(rank, world, port, out_path):
    import torch

    dist = _init(rank, world, port)
    p = _problem()
    y = workloads.gaussian(62, p.M)
    nd, nl = p.n_det, p.n_lambda
    g = np.zeros(p.n_chrom * p.grid.N)
    for c in shard.chunks_of_rank(rank, world, N_LAMBDA):  # one wavelength per chunk
        rs, rd = osolve.fields_splu(p, [c])
        ys = np.array([y[(s * nd + d) * nl + c] for s in range(p.n_src) for d in range(nd)])
        g += oborn.apply_T(p, rs, rd, ys, [c])
    gt = shard.allreduce_gradient(torch.tensor(g))
    if rank == 0:
        np.save(out_path, gt.numpy())
    dist.destroy_process_group()


def _failing_worker(rank, world, port, out_path):
    import torch

    dist = _init(rank, world, port)
    if rank == 1:
        os._exit(3)  # this rank dies between steps, before the collective
    try:
        shard.allreduce_gradient(torch.ones(16))
        result = "completed"
    except Exception as e:  # the peer's failure surfaces as an error on the survivor
        result = "error: " + type(e).__name__
    with open(out_path, "w") as f:
        f.write(result)
    os._exit(0)


def _run(target, world, out_path, timeout=120):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, out_path)) for r in range(world)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(timeout)
    alive = [q for q in procs if q.is_alive()]
    for q in alive:
        q.kill()
    return [q.exitcode for q in procs], bool(alive)


def test_chunks_partition_and_steps_distinct():
    for world in (1, 2, 3, 8):
        owned = [shard.chunks_of_rank(r, world, 8) for r in range(world)]
        flat = sorted(c for o in owned for c in o)
        assert flat == list(range(8))
        for step in range(5):
            chunks = [shard.chunk_of_step(step, r, world, 8) for r in range(world)]
            assert len(set(chunks)) == min(world, 8)


def test_sharded_gradient_equals_full_gradient(tmp_path):
    out = str(tmp_path / "g.npy")
    codes, hung = _run(_gradient_worker, 2, out)
    assert not hung and codes == [0, 0]
    p = _problem()
    rs, rd = osolve.fields_splu(p)
    g_full = oborn.apply_T(p, rs, rd, workloads.gaussian(62, p.M))
    g = np.load(out)
    assert np.abs(g - g_full).max() <= 1e-12 * np.abs(g_full).max()


def test_failed_rank_is_detected_not_hung(tmp_path):
    out = str(tmp_path / "result.txt")
    codes, hung = _run(_failing_worker, 2, out, timeout=90)
    assert not hung
    assert codes[1] == 3
    with open(out) as f:
        assert f.read().startswith("error")

"""Multi-rank path on CPU: world_size-2 gloo process groups.  Each rank
computes its shard with the oracle; the gathered shards must equal the full
oracle result bit for bit (the shards compute the same per-element sums)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_20347_gb300 import partition, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, result_path):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if kind == "2d":
            p = synth.uniform_problem(300, 520, 90, seed=40, alpha=0.5, beta=2.0)
            blk = partition.partition_2d(p.m, p.n, world)[rank]
            part = np.zeros((p.m, p.n))
            if not blk.empty:
                rows = np.arange(blk.row0, blk.row1)
                sub = oracle.gemm(p.A, p.B[:, blk.col0:blk.col1], p.C[:, blk.col0:blk.col1], p.alpha, p.beta,
                                  rows=rows)
                part[blk.row0:blk.row1, blk.col0:blk.col1] = sub
            t = torch.from_numpy(part)
            dist.all_reduce(t)          # blocks are disjoint: the sum assembles C
            if rank == 0:
                np.save(result_path, t.numpy())
        else:
            shapes = synth.grouped_shapes(40, seed=41, lo=4, hi=64)
            mine = partition.assign_problems(shapes, world)[rank]
            flat = []
            for i, (m, n, k) in enumerate(shapes):
                if i in mine:
                    q = synth.uniform_problem(m, n, k, seed=100 + i)
                    flat.append(oracle.gemm(q.A, q.B).ravel())
                else:
                    flat.append(np.zeros(m * n))
            t = torch.from_numpy(np.concatenate(flat))
            dist.all_reduce(t)
            if rank == 0:
                np.save(result_path, t.numpy())
    finally:
        dist.destroy_process_group()


def _run(kind, tmp_path, world=2):
    import oracle
    oracle.build()
    out = str(tmp_path / f"{kind}.npy")
    mp.start_processes(_worker, args=(world, _free_port(), kind, out), nprocs=world, join=True,
                       start_method="spawn")
    return np.load(out)


def test_partition_2d_covers_c_once():
    for (m, n, world) in [(300, 520, 2), (1000, 64, 4), (16384, 16384, 8), (5, 7, 3), (128, 128, 6)]:
        blocks = partition.partition_2d(m, n, world)
        assert len(blocks) == world
        cover = np.zeros((m, n), int)
        for b in blocks:
            cover[b.row0:b.row1, b.col0:b.col1] += 1
            for cut in (b.row0, b.col0):
                assert cut % partition.TILE == 0     # no tile straddles two ranks
        assert np.all(cover == 1)


def test_assign_problems_lpt():
    shapes = synth.grouped_shapes(1000, seed=0)
    owned = partition.assign_problems(shapes, 8)
    assert sorted(i for o in owned for i in o) == list(range(1000))
    loads = [sum(2.0 * shapes[i][0] * shapes[i][1] * shapes[i][2] for i in o) for o in owned]
    assert max(loads) / min(loads) < 1.05        # balanced within 5%


def test_gloo_two_ranks_2d_partition(tmp_path):
    import oracle
    got = _run("2d", tmp_path)
    p = synth.uniform_problem(300, 520, 90, seed=40, alpha=0.5, beta=2.0)
    assert np.array_equal(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta))


def test_gloo_two_ranks_grouped(tmp_path):
    import oracle
    got = _run("grouped", tmp_path)
    shapes = synth.grouped_shapes(40, seed=41, lo=4, hi=64)
    want = []
    for i, (m, n, k) in enumerate(shapes):
        q = synth.uniform_problem(m, n, k, seed=100 + i)
        want.append(oracle.gemm(q.A, q.B).ravel())
    assert np.array_equal(got, np.concatenate(want))

"""Multi-rank path on CPU (gloo, world size 2): each rank solves its own
slice of the batch and the gathered outputs equal the single-process solve.
The per-rank solver here is the FP64 oracle (the GPU kernels need a GPU);
what is under test is the partition and the gather."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2501_11592_gb300.shard import shard_range


def test_shard_range_partitions():
    for B in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            got = [shard_range(B, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == B
            assert all(got[i][1] == got[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
    # whole images of W columns
    for images, W, world in ((7, 4, 2), (64, 256, 8), (3, 5, 4), (0, 3, 2)):
        got = [shard_range(images * W, r, world, unit=W) for r in range(world)]
        assert got[0][0] == 0 and got[-1][1] == images * W
        assert all(b % W == 0 and e % W == 0 for b, e in got)
        counts = [(e - b) // W for b, e in got]
        assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 0, 2, unit=4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker_images(rank, world, port, q, unit):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads
    from paper_2501_11592_gb300.shard import gather_rows, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = workloads.random_problem(24, 60, 15, 4, seed=4, snr_db=30.0)
    b, e = shard_range(p.B, rank, world, unit=unit)
    o = oracle.clomp(p.A, p.Y[:, b:e], p.k, steps=20, tv_weight=0.5, image_width=3)
    coef = gather_rows(torch.from_numpy(o["coef"]), p.B, world, unit=unit)
    if rank == 0:
        q.put(coef.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _run(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for pr in procs:
        pr.start()
    out = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return out


def test_two_rank_image_shards_keep_images_whole():
    """Five images of three columns with the image prior: slices of whole
    images (unit = 3: 9 + 6 columns) reproduce the single-process solve; the
    column split 8 + 7 would cut the third image and change its columns."""
    import oracle
    import workloads
    p = workloads.random_problem(24, 60, 15, 4, seed=4, snr_db=30.0)
    ref = oracle.clomp(p.A, p.Y, p.k, steps=20, tv_weight=0.5, image_width=3)
    assert shard_range(15, 0, 2, unit=3) == (0, 9) and shard_range(15, 0, 2) == (0, 8)
    coef = _run(_worker_images, 2, 3)
    assert np.array_equal(coef, ref["coef"])
    # the cut image: its columns 6, 7 alone (a 2-column image) and 8 alone
    cut = oracle.clomp(p.A, p.Y[:, 6:8], p.k, steps=20, tv_weight=0.5, image_width=2)
    assert not np.array_equal(cut["coef"], ref["coef"][6:8])


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads
    from paper_2501_11592_gb300.shard import gather_rows, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = workloads.random_problem(24, 60, 9, 4, seed=3, snr_db=40.0)
    b, e = shard_range(p.B, rank, world)
    o = oracle.omp(p.A, p.Y[:, b:e], p.k)
    sup = gather_rows(torch.from_numpy(o["support"]), p.B, world)
    coef = gather_rows(torch.from_numpy(o["coef"]), p.B, world)
    if rank == 0:
        q.put((sup.numpy(), coef.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_solve_matches_single_process():
    import oracle
    import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    sup, coef = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = workloads.random_problem(24, 60, 9, 4, seed=3, snr_db=40.0)
    ref = oracle.omp(p.A, p.Y, p.k)
    assert np.array_equal(sup, ref["support"])
    assert np.array_equal(coef, ref["coef"])

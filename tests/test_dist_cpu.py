"""Host logic of the N-GPU bench on CPU: two gloo ranks (the path runs one
independent replica per GPU, so the only cross-rank step is the max over the
ranks' step times)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_setup()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        got = bench.max_over_ranks(1.5 + rank, w, torch.device("cpu"))
        # every replica gets its own image, seeded by its rank
        from paper_cs_0103001_gb300 import synth

        img = synth.sky(64, 64, 10, 3, r)
        digest = float(img.astype("float64").sum())
        ds = [None] * w
        dist.all_gather_object(ds, digest)
        q.put((r, w, local, got, ds))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_distinct_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, w, local, got, ds) in enumerate(out):
        assert (rank, w, local) == (r, world, r)
        assert got == pytest.approx(1.5 + world - 1)  # the slowest rank's time
        assert len(set(ds)) == world  # replicas process different images
    assert out[0][4] == out[1][4]


def test_single_rank_is_identity(monkeypatch):
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(2.25, 1, None) == 2.25


def _grad_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_cs_0103001_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B, n = 4, 64
        img = np.stack([synth.sky(n, n, 10, 7, b) for b in range(B)])
        G = synth.real_uniform((B, n, n), 8)
        H = synth.random_filter(n, n, 9)
        lo, hi = rank * B // world, (rank + 1) * B // world  # this rank's images
        _, gh = oracle.pipeline_grad(img[lo:hi], H, G[lo:hi])
        t = torch.from_numpy(np.ascontiguousarray(gh))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)  # the one collective of a data-parallel adjoint
        _, full = oracle.pipeline_grad(img, H, G)
        q.put((rank, float(np.abs(t.numpy() - full).max() / np.abs(full).max())))
    finally:
        dist.destroy_process_group()


def test_data_parallel_filter_gradient_is_one_sum():
    """The adjoint over a batch split across ranks: each rank's grad_H covers
    its own images, and one all-reduce sum gives the whole batch's (the
    filter gradient is a sum over images); two gloo ranks on CPU."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_grad_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(err <= 1e-12 for _, err in out)

"""Row-slab decomposition of one image over ranks, host side (no GPU).

The index maps of paper_cs_0103001_gb300.slab (which rows, slots and columns a
rank owns, where an element sits in each exchange buffer) are checked by
brute force, and the exchange itself runs on 2 and 4 gloo ranks on CPU: every
element of every rank's send buffer is tagged with its global (column, slot),
and after the all-to-all each rank must find, at the address its column pass
reads, exactly the slot of its column that the address stands for; the
exchange back must restore every rank's own slots."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_cs_0103001_gb300 import slab

CASES = [(512, 64, 2), (2048, 32, 4), (4096, 4096, 2), (512, 1024, 4), (1024, 2048, 8), (8192, 512, 2),
         (4096, 1024, 16)]


def test_rows_partition_and_pairs():
    for rows, cols, R in CASES:
        slab.check(rows, cols, R)
        owned = [x for r in range(R) for x in slab.slab_rows(rows, R, r)]
        assert sorted(owned) == list(range(rows))  # every row exactly once
        for r in range(R):
            mine = slab.slab_rows(rows, R, r)
            P = len(mine) // 2
            for i, p in enumerate(slab.pair_range(rows, R, r)):
                assert (mine[i], mine[P + i]) == slab.rows_of_pair(p, rows)
        cols_owned = [slab.column_block(cols, R, r) for r in range(R)]
        assert [kb for kb, _ in cols_owned] == [r * (cols // (2 * R)) for r in range(R)]
        assert sum(c for _, c in cols_owned) == cols // 2


def test_rank_slots_are_contiguous_runs_of_each_column():
    for rows, cols, R in CASES:
        g = min(slab.pairs_per_block(cols), rows // 2)
        lg = g.bit_length() - 1
        L = rows // R
        seen = set()
        for r in range(R):
            s = sorted(slab.slot_of_row(x, rows, lg) for x in slab.slab_rows(rows, R, r))
            assert s == list(range(r * L, (r + 1) * L))
            seen.update(s)
        assert seen == set(range(rows))


def test_invalid_decompositions_are_rejected():
    with pytest.raises(ValueError):
        slab.check(4096, 4096, 3)
    with pytest.raises(ValueError):
        slab.check(128, 128, 2)  # 32 pairs per rank, blocks of 64 pairs
    with pytest.raises(ValueError):
        slab.check(4096, 4, 4)  # no column for some ranks
    with pytest.raises(ValueError):
        slab.check(8, 8, 2)  # 2 pairs per rank, blocks of 4 pairs


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, rows, cols, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = rows // world
        half = cols // 2
        # send buffer as the forward row pass leaves it: [M/2][L], global slot r L + s
        k = torch.arange(half, dtype=torch.float64)[:, None]
        s = torch.arange(L, dtype=torch.float64)[None, :]
        tag = k * rows + rank * L + s
        send = torch.complex(tag, -tag).to(torch.complex64).reshape(-1).contiguous()
        recv = torch.empty_like(send)
        slab.exchange(send, recv)
        kbase, C = slab.column_block(cols, world, rank)
        bad = 0
        for kl in range(C):
            for g in range(rows):  # every global slot of every local column
                v = recv[slab.recv_offset(kl, g, rows, cols, world)]
                bad += int(v.real.item() != (kbase + kl) * rows + g or v.imag.item() != -v.real.item())
        back = torch.empty_like(send)
        slab.exchange(recv, back)
        same = bool(torch.equal(back, send))
        for kk in (0, half - 1):
            bad += int(back[slab.send_offset(kk, L - 1, rows, world)].real.item() != kk * rows + rank * L + L - 1)
        q.put((rank, bad, same))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,rows,cols", [(2, 16, 64), (4, 64, 32)])
def test_exchange_on_gloo_ranks(world, rows, cols):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, rows, cols, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == list(range(world))
    for rank, bad, same in out:
        assert bad == 0, f"rank {rank}: {bad} misplaced elements"
        assert same, f"rank {rank}: the exchange back did not restore its slots"

"""Host logic of one lattice split into strips over ranks, on CPU (gloo).

The CUDA library does the arithmetic of each strip; what runs on the host is
the partition of the rows and the per-step exchange (the neighbours' rows
across each cut, the per-particle force sums over ranks).  These tests run
that exchange over gloo with 2 and 3 CPU ranks, with host byte buffers in
place of the library's device buffers: every rank's rows reach the right
neighbour's halo (periodic and closed y axes, including two strips on a
periodic axis, where both messages travel between the same pair of ranks),
and the force sums are the same on every rank.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2106_08950_gb300 import strips as S   # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("ny,n", [(2000, 2), (2000, 3), (4096, 8), (100, 4), (18, 2), (8, 1)])
def test_strip_rows_cover_the_lattice_on_tile_boundaries(ny, n):
    rows = [S.strip_rows(ny, n, r) for r in range(n)]
    assert rows[0][0] == 0 and rows[-1][1] == ny
    for (a0, a1), (b0, b1) in zip(rows, rows[1:]):
        assert a1 == b0
    for y0, y1 in rows:
        assert y0 % 8 == 0 and (y1 % 8 == 0 or y1 == ny) and y1 - y0 >= 2
    tiles = [(y1 - y0 + 7) // 8 for y0, y1 in rows]
    assert max(tiles) - min(tiles) <= 1          # balanced to one tile row


def test_strip_rows_refuse_too_many_ranks():
    with pytest.raises(ValueError):
        S.strip_rows(20, 4, 0)                    # 3 tile rows over 4 ranks
    with pytest.raises(ValueError):
        S.strip_rows(17, 3, 2)                    # the last strip would hold 1 row


def test_neighbours():
    assert S.neighbours(0, 3, False) == (None, 1)
    assert S.neighbours(2, 3, False) == (1, None)
    assert S.neighbours(0, 3, True) == (2, 1)
    assert S.neighbours(1, 2, True) == (0, 0)


def rank_main(rank, world, port, periodic, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    row = 48
    # what each rank would hand over: its first row (south) and last row (north)
    send_s = torch.full((row,), 10 * rank + 1, dtype=torch.uint8)
    send_n = torch.full((row,), 10 * rank + 2, dtype=torch.uint8)
    recv_s = torch.zeros(row, dtype=torch.uint8)
    recv_n = torch.zeros(row, dtype=torch.uint8)
    fpart = torch.arange(10, dtype=torch.float64) * (rank + 1)
    ex = S.Exchange(fpart, send_s, send_n, recv_s, recv_n, periodic_y=periodic)
    ex.run()
    q.put((rank, recv_s.numpy().copy(), recv_n.numpy().copy(), fpart.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_exchange_over_gloo(world, periodic):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, rs, rn, fp = q.get(timeout=120)
        res[r] = (rs, rn, fp)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = np.arange(10) * sum(r + 1 for r in range(world))
    for r in range(world):
        rs, rn, fp = res[r]
        south, north = S.neighbours(r, world, periodic)
        # the south halo holds the south neighbour's last row, the north halo
        # the north neighbour's first row; a physical side receives nothing
        assert (rs == (10 * south + 2 if south is not None else 0)).all()
        assert (rn == (10 * north + 1 if north is not None else 0)).all()
        assert np.array_equal(fp, total)

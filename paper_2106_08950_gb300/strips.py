"""One lattice decomposed into horizontal strips, one per rank.

Every rank runs the procedure of Sec. 2.3 on its rows ``[y0, y1)`` of the
lattice (``dilbm_create_strip``) with a copy of every particle.  Two things
cross a cut each step, and this module moves them with ``torch.distributed``
(NCCL on the device buffers, or gloo through host copies):

* pull streaming (Eq. 13) at a strip's first and last rows needs the
  neighbour's post-collision row beside it (the three populations that cross
  the cut; the whole row of all nine planes is sent);
* the force and torque of Eqs. 18-19 and the Wan-Turek repulsion of Eq. 28
  are sums over nodes: each rank sums its own nodes and the per-particle
  sums are added over ranks (one all-reduce of 5 doubles per particle)
  before the rigid-body update of Eqs. 22-24, which every rank applies alike.

Strip cuts lie on multiples of 8 rows, the binning tiles' height, so each
tile belongs to one rank.  The CUDA library does all of the arithmetic; this
module only partitions and moves bytes.
"""
from __future__ import annotations

from typing import Optional, Tuple

TILE_ROWS = 8          # strip cuts lie on the binning tiles' row boundaries


def strip_rows(ny: int, nranks: int, rank: int) -> Tuple[int, int]:
    """Rows [y0, y1) of ``rank``'s strip: the ceil(ny / 8) tile rows dealt
    out as evenly as possible, the first ranks taking one more; raises
    ValueError where a strip would hold fewer than two rows."""
    tiles = (ny + TILE_ROWS - 1) // TILE_ROWS
    if nranks < 1 or not 0 <= rank < nranks or tiles < nranks:
        raise ValueError(f"cannot split {ny} rows ({tiles} tile rows) over {nranks} ranks")
    per, extra = divmod(tiles, nranks)
    t0 = rank * per + min(rank, extra)
    t1 = t0 + per + (1 if rank < extra else 0)
    y0, y1 = t0 * TILE_ROWS, min(t1 * TILE_ROWS, ny)
    if y1 - y0 < 2:
        raise ValueError(f"strip {rank} of {nranks} over {ny} rows would hold {y1 - y0} row(s)")
    return y0, y1


def neighbours(rank: int, nranks: int, periodic_y: bool) -> Tuple[Optional[int], Optional[int]]:
    """(south, north) neighbour ranks; None across a physical side."""
    south = rank - 1 if rank > 0 else (nranks - 1 if periodic_y else None)
    north = rank + 1 if rank < nranks - 1 else (0 if periodic_y else None)
    return south, north


class _DeviceBytes:
    """A device allocation of the CUDA library seen as a byte array, for
    torch.as_tensor (shares the memory; nothing is copied)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_bytes(ptr: int, nbytes: int):
    import torch
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")


class Exchange:
    """The per-step exchange of one strip.

    ``fpart`` (float64, np x 5) is summed over all ranks in place;
    ``recv_south`` <- the south neighbour's ``send_north`` and ``recv_north``
    <- the north neighbour's ``send_south`` (byte tensors of one row of nine
    planes each).  Device tensors under a gloo group go through host copies
    (after the library's stream has reached the exchange); under NCCL the
    collectives are queued on ``stream`` behind the library's work."""

    def __init__(self, fpart, send_south, send_north, recv_south, recv_north, periodic_y: bool,
                 group=None, stream=None, nparticles: Optional[int] = None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)
        self.south, self.north = neighbours(self.rank, self.nranks, periodic_y)
        self.stream = stream
        self.nparticles = nparticles
        self.dev = [fpart, send_south, send_north, recv_south, recv_north]
        self.staged = dist.get_backend(group) == "gloo" and fpart.is_cuda
        if self.staged:
            self.host = [t.detach().to("cpu").pin_memory() for t in self.dev]
        else:
            self.host = self.dev

    def _peer(self, r: int) -> int:
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def run(self) -> None:
        import torch
        dist = self.dist
        if self.staged:
            self.stream.synchronize()
            for k in (0, 1, 2):
                self.host[k].copy_(self.dev[k])
        fpart, send_s, send_n, recv_s, recv_n = self.host
        ctx = torch.cuda.stream(self.stream) if (self.stream is not None and not self.staged) else _Null()
        with ctx:
            if self.nparticles != 0:
                dist.all_reduce(fpart, op=dist.ReduceOp.SUM, group=self.group)
            # every rank issues its sends northward data first, then southward
            # data, and receives in the matching order, so that two messages
            # between the same pair of ranks (two strips on a periodic axis)
            # cannot be confused
            ops = []
            if self.north is not None:
                ops.append(dist.P2POp(dist.isend, send_n, self._peer(self.north), self.group, tag=0))
            if self.south is not None:
                ops.append(dist.P2POp(dist.isend, send_s, self._peer(self.south), self.group, tag=1))
            if self.south is not None:
                ops.append(dist.P2POp(dist.irecv, recv_s, self._peer(self.south), self.group, tag=0))
            if self.north is not None:
                ops.append(dist.P2POp(dist.irecv, recv_n, self._peer(self.north), self.group, tag=1))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
        if self.staged:
            with torch.cuda.stream(self.stream):
                for k in (0, 3, 4):
                    self.dev[k].copy_(self.host[k], non_blocking=True)


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class DecomposedSimulation:
    """One DI-LBM lattice split over the ranks of ``group`` (one process per
    GPU, or several processes sharing one GPU under gloo); every rank calls
    the same methods in the same order."""

    def __init__(self, prob, group=None, storage: str = "fp32", stream=None):
        import torch
        import torch.distributed as dist
        from . import dilbm as D
        from . import workloads as W
        self.prob = prob
        self.group = group
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)
        self.torch_stream = stream if stream is not None else torch.cuda.Stream()
        self.y0, self.y1 = strip_rows(prob.ny, self.nranks, self.rank)
        self.sim = D.Strip(prob, self.y0, self.y1, storage, int(self.torch_stream.cuda_stream))
        fpart, ss, sn, rs, rn, row_elems = self.sim.buffers()
        elem = 4 if storage == "fp32" else 2
        npart = len(prob.particles)
        t_f = device_bytes(fpart, 8 * 5 * max(1, npart)).view(torch.float64)
        rows = [device_bytes(p, elem * row_elems) for p in (ss, sn, rs, rn)]
        self.exchange = Exchange(t_f, *rows, periodic_y=prob.south.kind == W.PERIODIC, group=group,
                                 stream=self.torch_stream, nparticles=npart)

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.sim.begin()
            self.exchange.run()
            self.sim.end()

    def sync(self) -> None:
        self.sim.sync()

    def forces(self):
        return self.sim.forces()

    def gather(self, local):
        """Concatenate every rank's rows of a (..., rows, nx) array, in rank
        order, on every rank (host arrays)."""
        import numpy as np
        import torch
        import torch.distributed as dist
        rows = self.y1 - self.y0
        most = max(strip_rows(self.prob.ny, self.nranks, r)[1] - strip_rows(self.prob.ny, self.nranks, r)[0]
                   for r in range(self.nranks))
        pad = np.zeros(local.shape[:-2] + (most, local.shape[-1]), dtype=np.float64)
        pad[..., :rows, :] = local
        t = torch.from_numpy(pad)
        if dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        out = [torch.zeros_like(t) for _ in range(self.nranks)]
        dist.all_gather(out, t, group=self.group)
        parts = []
        for r, o in enumerate(out):
            a, b = strip_rows(self.prob.ny, self.nranks, r)
            parts.append(o.cpu().numpy()[..., : b - a, :])
        return np.concatenate(parts, axis=-2)

    def fields(self):
        """rho, ux, uy, phi of the whole lattice (every rank)."""
        return tuple(self.gather(a.astype("float64")) for a in self.sim.fields())

    def populations(self):
        return self.gather(self.sim.populations())

    def close(self) -> None:
        self.sim.close()

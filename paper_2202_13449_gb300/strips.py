"""Row-strip decomposition of one mesh over ranks (one GPU per rank).

The explicit step of Section 3.2 reads each cell's neighbours up to two
cells away (a face needs the Eq. 55 gradients of its two cells, a gradient
the Eq. 56 values around its cell), so a strip of rows j0 <= j < j1 takes
exactly the whole mesh's step once it holds the two rows beyond each inner
side as they were after the previous step.  This module holds the host
side of that decomposition:

* ``split_rows`` / ``neighbours`` -- which rows a rank owns, who borders it;
* ``StripExchange`` -- the halo exchange before every step, through
  ``torch.distributed`` point-to-point messages: host planes (gloo, or any
  backend) or the strips' device records (NCCL), each message stamped with
  the step and side so that a lost or misordered halo is an error
  (``HaloLost``) and never a silent wrong step;
* ``global_residual`` -- the whole mesh's R12 residual from every strip's
  residual sums (one all-reduce of four FP64 numbers);
* ``global_sum`` -- the whole mesh's Nusselt numbers from the strips'
  shares.

A strip is a ``capi.Solver`` created with ``rows=(j0, j1)``; the exchange
only needs its ``strip_get_rows`` / ``strip_set_halo`` (host mode) or
``strip_rows`` / ``strip_pack`` / ``strip_unpack`` (device mode).
"""
from __future__ import annotations

import datetime
import math

import numpy as np

SOUTH, NORTH = 2, 3  # the library's side numbers


class HaloLost(RuntimeError):
    """A neighbour's halo rows for a step did not arrive (or arrived for
    another step or side): the step must not be taken."""


def split_rows(ny: int, parts: int):
    """Row ranges [(j0, j1), ...] of `parts` strips covering 0..ny, sizes
    differing by at most one row, each at least 2 rows (a strip's halo is
    two rows deep)."""
    if parts < 1 or ny < 2 * parts:
        raise ValueError(f"{ny} rows cannot make {parts} strips of at least 2 rows")
    base, extra = divmod(ny, parts)
    out, j = [], 0
    for k in range(parts):
        n = base + (1 if k < extra else 0)
        out.append((j, j + n))
        j += n
    return out


def neighbours(rank: int, world: int):
    """(south rank or None, north rank or None) of strip `rank`: the mesh's
    own south and north sides are walls, not neighbours."""
    return (rank - 1 if rank > 0 else None, rank + 1 if rank < world - 1 else None)


class StripExchange:
    """Halo exchange of one rank's strip with its neighbours.

    ``mode="host"``: halo planes (4 x 2 x nx FP64) travel as CPU tensors
    (gloo) -- every backend works, the state crosses the host.
    ``mode="device"``: the strips' device records travel as CUDA byte
    tensors (NCCL), packed and unpacked on the device by the library; the
    current state buffer after k steps from a state upload is k % 2.

    Messages: a header (step, side the sender packed, sender rank) in front
    of the payload; ``timeout_s`` bounds each wait.
    """

    HEADER = 3

    def __init__(self, rank: int, world: int, nx: int, mode: str = "host",
                 timeout_s: float = 30.0, group=None, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank, self.world, self.nx = rank, world, nx
        self.mode = mode
        self.timeout = datetime.timedelta(seconds=timeout_s)
        self.group = group
        self.device = device
        self.south, self.north = neighbours(rank, world)
        self.drop = None  # tests: (step, side) whose message this rank does not send
        self._bufs = {}

    # -- message buffers
    def _buf(self, key, n, dtype):
        t = self._bufs.get(key)
        if t is None or t.numel() != n or t.dtype != dtype:
            dev = self.device if self.mode == "device" else "cpu"
            t = self.torch.empty(n, dtype=dtype, device=dev)
            self._bufs[key] = t
        return t

    def _header(self, step: int, side: int):
        return np.array([float(step), float(side), float(self.rank)])

    def _check(self, head, step: int, side: int, src: int):
        h = [float(x) for x in head]
        if h[0] != float(step) or h[1] != float(side) or h[2] != float(src):
            raise HaloLost(f"rank {self.rank}: halo from rank {src} carries step {h[0]:.0f}, "
                           f"side {h[1]:.0f}, sender {h[2]:.0f}; expected step {step}, side "
                           f"{side}, sender {src}")

    def exchange(self, strip, step: int, buffer: int | None = None):
        """Send this strip's boundary rows to its neighbours and set the rows
        they send as its halos, for the step about to be taken (`step` = the
        number of steps taken so far; in device mode `buffer` = the current
        state buffer, step % 2 by default).  Raises HaloLost if a neighbour's
        rows do not arrive within the timeout or belong to another step."""
        dist = self.dist
        ops, recvs = [], []
        # my south rows go to the south neighbour (its north halo), and so
        # on; sends and receives go out as one batch (no ordering deadlock)
        for side, peer in ((SOUTH, self.south), (NORTH, self.north)):
            if peer is None:
                continue
            out = self._pack(strip, side, step, buffer)
            if self.drop is not None and tuple(self.drop) == (step, side):
                continue  # injected loss: the neighbour's wait must run out
            ops.append(dist.P2POp(dist.isend, out, peer, group=self.group))
        for side, peer in ((SOUTH, self.south), (NORTH, self.north)):
            if peer is None:
                continue
            inb = self._recv_buf(strip, side)
            ops.append(dist.P2POp(dist.irecv, inb, peer, group=self.group))
            recvs.append((side, peer, inb))
        works = dist.batch_isend_irecv(ops) if ops else []
        for w in works:
            try:
                ok = w.wait(timeout=self.timeout)
            except RuntimeError as e:  # the backend's own timeout
                raise HaloLost(f"rank {self.rank}: a halo for step {step} did not arrive "
                               f"within {self.timeout.total_seconds():.0f} s ({e})") from None
            if ok is False:
                raise HaloLost(f"rank {self.rank}: a halo for step {step} did not arrive")
        for side, peer, inb in recvs:
            # the neighbour packed the side facing me
            self._unpack(strip, side, step, buffer, inb, peer, NORTH if side == SOUTH else SOUTH)

    # -- host planes
    def _pack(self, strip, side, step, buffer):
        if self.mode == "device":
            _, nbytes = strip.strip_rows(side, False, 0)
            # the header travels as its own 8-byte words in front of the records
            out = self._buf(("out", side), 8 * self.HEADER + nbytes, self.torch.uint8)
            head = self.torch.from_numpy(self._header(step, side).view(np.uint8).copy())
            out[: 8 * self.HEADER].copy_(head)
            b = step % 2 if buffer is None else buffer
            self.torch.cuda.current_stream().synchronize()  # the header copy
            strip.strip_pack(side, b, out.data_ptr() + 8 * self.HEADER)
            strip.sync()  # the records, on the library's stream
            return out
        rows = np.asarray(strip.strip_get_rows(side), dtype=np.float64).reshape(-1)
        out = self._buf(("out", side), self.HEADER + rows.size, self.torch.float64)
        out[: self.HEADER] = self.torch.from_numpy(self._header(step, side))
        out[self.HEADER:] = self.torch.from_numpy(rows)
        return out

    def _recv_buf(self, strip, side):
        if self.mode == "device":
            _, nbytes = strip.strip_rows(side, True, 0)
            return self._buf(("in", side), 8 * self.HEADER + nbytes, self.torch.uint8)
        return self._buf(("in", side), self.HEADER + 8 * self.nx, self.torch.float64)

    def _unpack(self, strip, side, step, buffer, inb, peer, peer_side):
        if self.mode == "device":
            head = inb[: 8 * self.HEADER].cpu().numpy().view(np.float64)
            self._check(head, step, peer_side, peer)
            b = step % 2 if buffer is None else buffer
            strip.strip_unpack(side, b, inb.data_ptr() + 8 * self.HEADER)
            strip.sync()
            return
        a = inb.numpy()
        self._check(a[: self.HEADER], step, peer_side, peer)
        strip.strip_set_halo(side, a[self.HEADER:].reshape(4, 2, self.nx))


def global_residual(sums, group=None):
    """(R_u, R_T) of the whole mesh from this rank's residual sums (4,)
    (rtlbfs_residual_sums): one all-reduce (sum) of the four FP64 sums, then
    R = sqrt(numerator) / sqrt(denominator) as R12 defines it (infinite for
    a zero denominator)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(sums, dtype=np.float64).reshape(4))
    if dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    s = t.cpu().numpy()

    def r(num, den):
        return math.sqrt(num) / math.sqrt(den) if den > 0 else math.inf

    return r(s[0], s[1]), r(s[2], s[3])


def global_sum(x: float, group=None) -> float:
    """Sum of a scalar share over the ranks (a strip's share of a Nusselt
    number: west, east, mid-plane and Eq. 69 sums add over strips)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.cpu()[0])

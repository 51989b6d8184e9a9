"""One long signal split by frame ranges over the ranks of a process group,
one GPU per rank (the C ABI's sst_part_* calls; Sec. 2.1: frames are
independent, and only the overlap-add of Eq. 26 couples neighbours).

Every rank holds a plan with the same parameters and the samples its frames
read.  The path has two exchanges, both small:

* the relative threshold needs max |S^g| over every frame: one all-reduce
  (max) of one float;
* the overlap-add segments of the tiles at each boundary go to the ranks
  whose output samples they cover (one segment of (B - 1) hop + L floats per
  boundary tile, 16 kB at Nf 4096).

The exchanges go through a small communicator object with two methods
(``allreduce_max(tensor)`` and ``exchange(sends, recvs)``); ``DistComm``
implements them with torch.distributed (NCCL between GPUs, plain point-to-
point sends of device buffers).  The layouts and the exchange lists are host
arithmetic.  Every step of the transform runs in libsst.so's kernels.
"""
from __future__ import annotations

from . import sst as S


def layouts(plan, parts: int) -> list:
    """The layout (dict) of every part of `plan`'s signal."""
    return [S.sst_part_layout(plan.handle, p, parts).as_dict() for p in range(parts)]


def exchange_lists(lays: list, me: int):
    """The tile ranges rank `me` sends and receives: (peer, first tile, end
    tile) triples.  A rank sends the tiles it computed that another rank's
    output samples need, and receives the tiles its own output needs from the
    ranks that computed them."""
    sends, recvs = [], []
    mine = lays[me]
    for q, lay in enumerate(lays):
        if q == me:
            continue
        # tiles I computed that q needs
        a, b = max(mine["tile_begin"], lay["need_begin"]), min(mine["tile_end"], lay["need_end"])
        if b > a:
            sends.append((q, a, b))
        # tiles q computed that I need
        a, b = max(lay["tile_begin"], mine["need_begin"]), min(lay["tile_end"], mine["need_end"])
        if b > a:
            recvs.append((q, a, b))
    return sends, recvs


def segments(workspace, ola_offset: int, seg_len: int, t0: int, t1: int):
    """The workspace's float32 view of the segments of tiles [t0, t1)."""
    import torch
    lo = ola_offset + 4 * seg_len * t0
    hi = ola_offset + 4 * seg_len * t1
    return workspace[lo:hi].view(torch.float32)


class DistComm:
    """The two exchanges over a torch.distributed process group.  With NCCL
    the device buffers are sent as they are; with a backend that moves host
    memory only (gloo), through host copies."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.host = dist.get_backend(group) == "gloo"

    def _stage(self, t):
        return t.cpu() if (self.host and t.is_cuda) else t

    def allreduce_max(self, t):
        h = self._stage(t)
        self.dist.all_reduce(h, op=self.dist.ReduceOp.MAX, group=self.group)
        if h is not t:
            t.copy_(h)

    def exchange(self, sends, recvs):
        """sends / recvs: (peer rank, tensor) pairs; all posted, then awaited."""
        hs = [(peer, self._stage(t)) for peer, t in sends]
        hr = [(peer, self._stage(t) if not self.host else t.new_empty(t.shape, device="cpu"), t)
              for peer, t in recvs]
        ops = [self.dist.P2POp(self.dist.isend, h, peer, group=self.group) for peer, h in hs]
        ops += [self.dist.P2POp(self.dist.irecv, h, peer, group=self.group) for peer, h, _ in hr]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        for _, h, t in hr:
            if h is not t:
                t.copy_(h)


def run(plan, x_part, rank: int, parts: int, comm, lays=None):
    """This rank's share of sst_forward_inverse without a TFR output: the
    reconstruction of its output samples [out_begin, out_end).  x_part holds
    the signal's samples [x_begin, x_end) of this rank's layout, on the
    plan's device."""
    import torch
    lays = lays if lays is not None else layouts(plan, parts)
    lay = lays[rank]
    part = S.sst_part(**lay)
    ws = plan.workspace
    r = torch.zeros(1, dtype=torch.float32, device=plan.device)
    S.sst_part_prepass(plan.handle, part, x_part, r, ws)
    comm.allreduce_max(r)
    S.sst_part_forward_inverse(plan.handle, part, x_part, r, ws)
    off, seg_len, _ = S.sst_part_segments(plan.handle)
    sends, recvs = exchange_lists(lays, rank)
    comm.exchange([(q, segments(ws, off, seg_len, a, b)) for q, a, b in sends],
                  [(q, segments(ws, off, seg_len, a, b)) for q, a, b in recvs])
    xhat = torch.empty(lay["out_end"] - lay["out_begin"], dtype=torch.float32, device=plan.device)
    S.sst_part_finalize(plan.handle, part, ws, xhat)
    return xhat

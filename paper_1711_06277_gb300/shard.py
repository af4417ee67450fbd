"""One trace split over the ranks of a process group by source (one GPU per rank).

Sources are independent and their deposits add (Sec. 2.1: several sources are handled by
summing over the rays of every source), so each rank holds the whole density field, traces a
disjoint subset of the sources, and one all-reduce (sum) of the per-cell outputs gives every
rank the full result:

* the subsets come from ``art_partition_sources`` (longest processing time first) over the
  per-source work estimates of ``art_estimate_work``, computed by rank 0 and broadcast;
* a trace sums gamma and the three force components in one (4, nz, ny, nx) float32 buffer
  (16 bytes per cell, the size of the per-cell accumulator) and the FP64 tallies in another;
* the reverse sweep sums dloss/dlog n_H0 per cell (4 bytes per cell); dloss/dL_s is computed
  by the rank that owns source s and summed into a zero-padded vector of all sources.

Everything here is argument marshalling and ``torch.distributed`` calls; the traces run in
the CUDA library. With a group of one rank it is the plain single-GPU trace.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch
import torch.distributed as dist

from . import _lib as C
from .art import Grid, Params

# per-trace tallies summed over ranks (FP64), in this order
TALLY_KEYS = ("crossings", "rays_total", "destroy", "L_in", "L_absorbed", "L_escaped",
              "L_dropped")


def partition(work, nranks: int):
    """Rank of every source and the summed estimate per rank (``art_partition_sources``)."""
    work = np.ascontiguousarray(np.asarray(work, dtype=np.float64).reshape(-1))
    rank = np.zeros(len(work), dtype=np.int32)
    load = np.zeros(nranks, dtype=np.float64)
    P = ctypes.POINTER
    C.check(C.lib().art_partition_sources(len(work), work.ctypes.data_as(P(ctypes.c_double)),
                                          int(nranks), rank.ctypes.data_as(P(ctypes.c_int)),
                                          load.ctypes.data_as(P(ctypes.c_double))),
            "art_partition_sources")
    return rank, load


def reduce_fields(buf: torch.Tensor, group=None) -> torch.Tensor:
    """Sums a per-rank output buffer over the ranks, in place (one all-reduce)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf


def reduce_tallies(stats: dict | None, device, group=None) -> dict:
    """Sums the per-rank tallies of ``TALLY_KEYS`` (a rank without sources passes None)."""
    vals = [float(stats[k]) if stats else 0.0 for k in TALLY_KEYS]
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    reduce_fields(t, group)
    out = dict(zip(TALLY_KEYS, t.tolist()))
    for k in ("crossings", "rays_total", "destroy"):
        out[k] = int(round(out[k]))
    return out


class ShardedTrace:
    """A trace of all ``pos``/``L`` sources split by source over the ranks of ``group``.

    Every rank passes the same field, sources and parameters. ``trace()`` returns gamma
    (nz, ny, nx) and force (3, nz, ny, nx) summed over the ranks, identical on every rank.
    """

    def __init__(self, nH0: torch.Tensor, dx: float, pos, L, params: Params, group=None,
                 lo=(0.0, 0.0, 0.0), nH: torch.Tensor | None = None,
                 stream: torch.cuda.Stream | None = None, work=None):
        self.group = group
        init = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if init else 0
        self.world = dist.get_world_size(group) if init else 1
        self.params = params
        self.pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
        self.L = np.asarray(L, dtype=np.float64).reshape(-1)
        self.device = nH0.device
        self.grid = Grid(nH0, dx, lo=lo, nH=nH, stream=stream)
        if self.world > 1:
            if work is None:
                est = torch.zeros(len(self.L), dtype=torch.float64, device=self.device)
                if self.rank == 0:
                    self.grid.add_sources(self.pos, self.L)
                    est.copy_(torch.from_numpy(self.grid.estimate_work(params)))
                    self.grid.clear_sources()
                dist.broadcast(est, src=0, group=group)
                work = est.cpu().numpy()
            self.rank_of, self.load = partition(work, self.world)
        else:
            self.rank_of = np.zeros(len(self.L), dtype=np.int32)
            self.load = np.array([float(np.sum(work))]) if work is not None else None
        self.mine = np.flatnonzero(self.rank_of == self.rank)
        if len(self.mine):
            self.grid.add_sources(self.pos[self.mine], self.L[self.mine])
        nz, ny, nx = self.grid.shape
        self.out = torch.empty((4, nz, ny, nx), dtype=torch.float32, device=self.device)

    def trace(self, stats: bool = True) -> dict:
        gamma, force = self.out[0], self.out[1:4]
        st = None
        if len(self.mine):
            r = self.grid.trace(self.params, force=True, stats=stats,
                                out={"gamma": gamma, "force": force})
            st = r["stats"]
        else:
            self.out.zero_()
        reduce_fields(self.out, self.group)
        res = {"gamma": gamma, "force": force, "local_stats": st, "sources": len(self.mine)}
        if stats:
            res["stats"] = reduce_tallies(st, self.device, self.group)
        return res

    def backward(self, w: torch.Tensor | None, v: torch.Tensor | None = None):
        """dloss/dlog n_H0 per cell and dloss/dL per source (all sources, float64) for
        loss = sum w gamma + sum v . force of the whole trace, on every rank."""
        grad = torch.zeros(self.grid.shape, dtype=torch.float32, device=self.device)
        dL = torch.zeros(len(self.L), dtype=torch.float64, device=self.device)
        if len(self.mine):
            g, dl, _ = self.grid.trace_backward(self.params, w, stats=False, v=v)
            grad.copy_(g)
            dL[torch.as_tensor(self.mine, device=self.device)] = dl
        reduce_fields(grad, self.group)
        reduce_fields(dL, self.group)
        return grad, dL

    def close(self):
        self.grid.close()

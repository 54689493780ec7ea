"""One system solved in shards: the paper's distributed dichotomy process (Sec. 2.4-2.5).

Shard k of S owns a contiguous range of whole windows of a bound plan and holds only its own rows
of F and x.  The library computes everything on the device (`dichotomy_shard_reduce`, `_bounds`,
`_finish`); what crosses shards is, first, the four numbers of each shard's composite prefix and
suffix maps of eq. 15's scans (an all-gather: the paper's All-to-One-Reduce levels of eq. 17-19
collapse to one level because the maps compose associatively), then one boundary value to each
neighbour.  The transport is the caller's: `solve_sharded` runs every shard in this process and passes the
messages through host memory; `Exchange` / `DistExchange` move them between processes (one per
shard) with `torch.distributed` collectives on host tensors.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check
from .dichotomy import _dev, _stream

__all__ = ["shard_info", "Shard", "Exchange", "DistExchange", "fold_maps", "neighbour_values", "solve_sharded"]


def shard_info(plan, nshards: int, k: int) -> dict:
    info = _lib.dich_shard_info()
    check(_lib.load().dichotomy_shard_info(plan.handle, int(nshards), int(k), ctypes.byref(info)),
          "dichotomy_shard_info")
    return {name: getattr(info, name) for name, _ in info._fields_}


def fold_maps(all_maps, k: int):
    """The prefix entering shard k and the suffix beyond it from every shard's (prefix a, b, suffix
    a, b), composed in shard order from zero at both ends of the system (the same fold the library
    does on the device in dichotomy_shard_bounds; here for checking the exchange)."""
    A = 0.0
    for j in range(k):
        A = all_maps[4 * j] * A + all_maps[4 * j + 1]
    B = 0.0
    for j in range(len(all_maps) // 4 - 1, k, -1):
        B = all_maps[4 * j + 2] * B + all_maps[4 * j + 3]
    return A, B


class Shard:
    """Shard k of S of a bound Plan: its rows, workspace and the three device steps."""

    def __init__(self, plan, nshards: int, k: int, device=None):
        self.plan, self.S, self.k = plan, int(nshards), int(k)
        self.info = shard_info(plan, nshards, k)
        dev = device if device is not None else plan.workspace.device
        self.ws = torch.empty(self.info["workspace_bytes"] + 256, dtype=torch.uint8, device=dev)
        self._ws = (self.ws.data_ptr() + 255) // 256 * 256
        self.rows = slice(self.info["row_lo"], self.info["row_hi"])

    def reduce(self, F: torch.Tensor, x: torch.Tensor, stream=None):
        out = (ctypes.c_double * 4)()
        check(_lib.load().dichotomy_shard_reduce(self.plan.handle, self.S, self.k, _dev(F, "F"), _dev(x, "x"),
                                                 ctypes.c_void_p(self._ws), self.info["workspace_bytes"], out,
                                                 _stream(stream)), "dichotomy_shard_reduce")
        return list(out)

    def bounds(self, all_maps, stream=None):
        m = (ctypes.c_double * (4 * self.S))(*[float(v) for v in all_maps])
        out = (ctypes.c_double * 2)()
        check(_lib.load().dichotomy_shard_bounds(self.plan.handle, self.S, self.k, m, ctypes.c_void_p(self._ws),
                                                 self.info["workspace_bytes"], out, _stream(stream)),
              "dichotomy_shard_bounds")
        return list(out)

    def finish(self, F: torch.Tensor, x: torch.Tensor, nbr, stream=None):
        v = (ctypes.c_double * 2)(float(nbr[0]), float(nbr[1]))
        check(_lib.load().dichotomy_shard_finish(self.plan.handle, self.S, self.k, _dev(F, "F"), _dev(x, "x"), v,
                                                 ctypes.c_void_p(self._ws), self.info["workspace_bytes"],
                                                 _stream(stream)), "dichotomy_shard_finish")


class Exchange:
    """How the shards' two messages travel: all_gather_maps(k, maps4) -> the 4 S numbers of every
    shard in order; neighbours(k, ends2) -> (x before the shard, x after it), zeros at the ends."""

    def all_gather_maps(self, k: int, maps4):
        raise NotImplementedError

    def neighbours(self, k: int, ends2):
        raise NotImplementedError


class DistExchange(Exchange):
    """One process per shard (rank k = shard k) over a torch.distributed process group: an
    all-gather of the 4 numbers, then an all-gather of the 2 boundary values, on host tensors
    (gloo) or device tensors (a backend that needs them)."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist, self.group, self.device = dist, group, device
        self.S = dist.get_world_size(group)

    def _gather(self, vals):
        t = torch.tensor(vals, dtype=torch.float64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.S)]
        self.dist.all_gather(out, t, group=self.group)
        return [o.cpu().tolist() for o in out]

    def all_gather_maps(self, k, maps4):
        return [v for m in self._gather(list(maps4)) for v in m]

    def neighbours(self, k, ends2):
        return neighbour_values(self._gather(list(ends2)), k)


def neighbour_values(ends, k: int):
    """What shard k receives from its neighbours' (x at first row, x at last row): the last value
    of shard k-1 and the first value of shard k+1, zeros at the system's ends."""
    return (ends[k - 1][1] if k > 0 else 0.0, ends[k + 1][0] if k + 1 < len(ends) else 0.0)


def solve_sharded(plan, F: torch.Tensor, nshards: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """x = T^-1 F with the system split into `nshards` shards in this process: each shard reads and
    writes only its own rows of F and x (views), the two exchanges go through host memory."""
    shards = [Shard(plan, nshards, k) for k in range(nshards)]
    x = torch.empty_like(F) if out is None else out
    all_maps = [v for s in shards for v in s.reduce(F[s.rows], x[s.rows], stream)]
    ends = [s.bounds(all_maps, stream) for s in shards]
    for s in shards:
        s.finish(F[s.rows], x[s.rows], neighbour_values(ends, s.k), stream)
    return x

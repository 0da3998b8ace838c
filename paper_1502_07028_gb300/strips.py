"""A PTCA sweep split over several ranks (one GPU each) by strips of the lattice.

The paper distributes the independent clusters of a block over processes
and, once the block is done, gathers the accepted updates on a master and
broadcasts the new configuration to every process before the next block
(Sec. III.b, Fig. 4).  Here the distribution is spatial and the exchange is
local:

* The lattice is cut into strips along its outermost axis (rows of a square
  lattice, planes of a cube, segments of a chain).  A rank owns the visits
  whose update site lies in one of its strips.  The block schedule halves
  every axis, so there each rank takes one strip in each half of the outer
  axis, and every stage keeps all ranks busy.
* A rank reads the windows of its own visits: its strips plus a halo of
  L_c - 1 rows (the window reaches o rows to one side of an update site and
  L_c - 1 - o to the other).  It keeps a full-size copy of the spins (24 bytes
  a site), of which only that region is kept up to date.
* After every stage each rank sends every other rank the spins, as they are
  after the stage, of its visits of that stage whose update sites lie in the
  other rank's windows, and writes what it receives.  A rejected proposal
  carries its unchanged spin, so the messages have fixed sizes that both sides
  know from the plan.

Every visit therefore reads the configuration it reads on one GPU, and draws
the same random numbers (they are keyed by sweep and site): the partitioned
sweep equals the single-domain sweep, decision for decision.

The plan (``StripPlan``) and the per-rank driver (``StripRank``) are host
logic.  The compute is a backend with three calls -- run some visits of a
stage, gather the spins of some sites, scatter spins into some sites --
which ``GpuStripBackend`` maps onto the library's ptca_stage_run,
ptca_get_sites and ptca_set_sites; the exchange is a callable, for example
``TorchDistExchange`` (NCCL between GPUs, or gloo).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .ptca import SCHEDULE_BLOCK, SCHEDULE_TILED, Config, ptca_get_sites, ptca_schedule, ptca_set_sites, \
    ptca_stage_run


def _axis_window(L: int, periodic: int, Lc: int, o: int, c: np.ndarray):
    """Window of update sites at coordinates c along one axis (the library's
    rule): periodic -> L_c sites from c - o, wrapped; open -> the same range
    clipped to [0, L).  Returns (start, extent) arrays."""
    if L == 1:
        return np.zeros_like(c), np.ones_like(c)
    a = c - o
    if periodic:
        return a % L, np.full_like(c, Lc)
    b = np.minimum(a + Lc - 1, L - 1)
    a = np.maximum(a, 0)
    return a, b - a + 1


def window_sites(cfg: Config, sites: np.ndarray) -> list[np.ndarray]:
    """Lattice sites of the window of each update site (Sec. II.b)."""
    Lz = max(cfg.Lz, 1)
    o = cfg.update_offset if cfg.update_offset >= 0 else (cfg.L_c // 2 if cfg.schedule == SCHEDULE_TILED else 0)
    sites = np.asarray(sites, dtype=np.int64)
    x, y, z = sites % cfg.Lx, (sites // cfg.Lx) % cfg.Ly, sites // (cfg.Lx * cfg.Ly)
    x0, ex = _axis_window(cfg.Lx, cfg.periodic, cfg.L_c, o, x)
    y0, ey = _axis_window(cfg.Ly, cfg.periodic, cfg.L_c, o if cfg.Ly > 1 else 0, y)
    z0, ez = _axis_window(Lz, cfg.periodic, cfg.L_c, o if Lz > 1 else 0, z)
    out = []
    for k in range(sites.size):
        xs = (x0[k] + np.arange(ex[k])) % cfg.Lx
        ys = (y0[k] + np.arange(ey[k])) % cfg.Ly
        zs = (z0[k] + np.arange(ez[k])) % Lz
        out.append(((zs[:, None, None] * cfg.Ly + ys[None, :, None]) * cfg.Lx + xs[None, None, :]).ravel())
    return out


@dataclass
class StripPlan:
    """Which rank runs which visit of each stage, and which spins each rank
    sends which other rank after each stage.

    owned[r][s]    update sites of stage s that rank r runs (schedule order)
    send[s][r][q]  the sites of owned[r][s] that lie in rank q's windows
    reads[r]       boolean mask over the sites: rank r's windows (strips + halo)
    strips[r]      (first, end) coordinate ranges of rank r's strips along the
                   outer axis"""
    cfg: Config
    world: int
    stages: list = field(default_factory=list)
    owned: list = field(default_factory=list)
    send: list = field(default_factory=list)
    reads: list = field(default_factory=list)
    strips: list = field(default_factory=list)

    @classmethod
    def build(cls, cfg: Config, world: int, strips_per_rank: int | None = None) -> "StripPlan":
        if world < 1:
            raise ValueError("world must be >= 1")
        Lz = max(cfg.Lz, 1)
        stages = [np.asarray(s, dtype=np.int32) for s in ptca_schedule(cfg)]  # validates cfg, no GPU
        N = cfg.Lx * cfg.Ly * Lz
        if Lz > 1:
            L_out, outer = Lz, lambda s: s // (cfg.Lx * cfg.Ly)
        elif cfg.Ly > 1:
            L_out, outer = cfg.Ly, lambda s: (s // cfg.Lx) % cfg.Ly
        else:
            L_out, outer = cfg.Lx, lambda s: s % cfg.Lx
        if strips_per_rank is None:
            strips_per_rank = 2 if cfg.schedule == SCHEDULE_BLOCK else 1
        n_strips = world * strips_per_rank
        if n_strips > L_out:
            raise ValueError(f"{n_strips} strips do not fit an outer extent of {L_out}")
        bounds = [(i * L_out) // n_strips for i in range(n_strips + 1)]
        owner_of_coord = np.empty(L_out, dtype=np.int32)
        strips = [[] for _ in range(world)]
        for i in range(n_strips):
            owner_of_coord[bounds[i]:bounds[i + 1]] = i % world
            strips[i % world].append((bounds[i], bounds[i + 1]))
        owner = owner_of_coord[outer(np.arange(N))]
        owned = [[s[owner[s] == r] for s in stages] for r in range(world)]
        reads = []
        for r in range(world):
            mask = np.zeros(N, dtype=bool)
            for s in owned[r]:
                for w in window_sites(cfg, s):
                    mask[w] = True
            reads.append(mask)
        send = [[[owned[r][s][reads[q][owned[r][s]]] if q != r else owned[r][s][:0] for q in range(world)]
                 for r in range(world)] for s in range(len(stages))]
        return cls(cfg=cfg, world=world, stages=stages, owned=owned, send=send, reads=reads, strips=strips)

    @property
    def n_stages(self) -> int:
        return len(self.stages)

    def halo_rows(self) -> int:
        """Depth of the halo around a strip along the outer axis: L_c - 1."""
        return self.cfg.L_c - 1


class StripRank:
    """One rank's side of a partitioned sweep: for every stage, run the owned
    visits, send the spins the others read, write the spins received."""

    def __init__(self, plan: StripPlan, rank: int, backend, exchange):
        self.plan, self.rank, self.backend, self.exchange = plan, rank, backend, exchange

    def run_stage(self, s: int, sweep_index: int):
        """The owned visits of stage s; returns the messages for the others."""
        p, r = self.plan, self.rank
        self.backend.run_visits(p.owned[r][s], sweep_index)
        return {q: self.backend.gather(p.send[s][r][q]) for q in range(p.world) if q != r and p.send[s][r][q].size}

    def expected(self, s: int):
        """Number of sites each other rank sends this rank after stage s."""
        p, r = self.plan, self.rank
        return {q: int(p.send[s][q][r].size) for q in range(p.world) if q != r and p.send[s][q][r].size}

    def finish_stage(self, s: int, received) -> None:
        for q, spins in received.items():
            self.backend.scatter(self.plan.send[s][q][self.rank], spins)

    def sweep(self, sweep_index: int) -> None:
        for s in range(self.plan.n_stages):
            out = self.run_stage(s, sweep_index)
            self.finish_stage(s, self.exchange(out, self.expected(s)))


class TorchDistExchange:
    """Point-to-point exchange of one stage's messages over torch.distributed
    (NCCL between GPUs with device tensors; gloo on the host).  out: {peer:
    float64 tensor (count, 3)}; expected: {peer: count}.  Returns {peer:
    tensor (count, 3)} on `device`."""

    def __init__(self, device="cpu", group=None):
        self.device, self.group = device, group

    def __call__(self, out, expected):
        import torch
        import torch.distributed as dist
        recv = {q: torch.empty((n, 3), dtype=torch.float64, device=self.device) for q, n in expected.items()}
        ops = [dist.P2POp(dist.irecv, t, q, group=self.group) for q, t in sorted(recv.items())]
        ops += [dist.P2POp(dist.isend, t.contiguous(), q, group=self.group) for q, t in sorted(out.items())]
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return recv


class GpuStripBackend:
    """The library as a strip backend: a context holding this rank's copy of
    the configuration; visits through ptca_stage_run, messages through
    ptca_get_sites / ptca_set_sites (device tensors, or host tensors when
    `device` is "cpu" for a host-side exchange)."""

    def __init__(self, ctx, device="cuda", stream=None):
        self.ctx, self.device, self.stream = ctx, device, stream

    def run_visits(self, sites, sweep_index: int) -> None:
        if len(sites):
            ptca_stage_run(self.ctx.h, sweep_index, sites, stream=self.stream)

    def gather(self, sites):
        import torch
        out = torch.empty((len(sites), 3), dtype=torch.float64, device=self.device)
        if len(sites):
            ptca_get_sites(self.ctx.h, sites, out, stream=self.stream)
        return out

    def scatter(self, sites, spins) -> None:
        if len(sites):
            ptca_set_sites(self.ctx.h, sites, spins.contiguous(), stream=self.stream)

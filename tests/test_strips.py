"""The lattice split over ranks by strips (paper Sec. III.b, Fig. 4: the
independent clusters of a block run on several processes, and the accepted
updates reach the others before the next block), on the host.

Two gloo ranks each run the visits of their strips, with the oracle as the
compute behind the same driver and exchange the GPU path uses, and swap the
spins of the halo after every stage.  Together they must reproduce the
oracle's sequential sweep bit for bit -- every F_old, F_new, ln u, decision
and final spin -- over several sweeps, on periodic and open lattices, with
the tiled and the paper's block schedules.  No GPU is involved."""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_1502_07028_gb300 as P  # noqa: E402
from paper_1502_07028_gb300 import strips  # noqa: E402

CASES = {
    # 8x8 torus, 4x4 clusters, tiled stride 4 (16 stages of 4, central site):
    "tiled_periodic": dict(Lx=8, Ly=8, L_c=4, stride=4, schedule=P.SCHEDULE_TILED, periodic=1, T=0.1),
    # the paper's block schedule (4 stages of 16, corner site), two strips per rank
    "block_periodic": dict(Lx=8, Ly=8, L_c=4, schedule=P.SCHEDULE_BLOCK, periodic=1, T=0.1),
    # 9x8 open lattice, 3x3 clusters clipped at the edges, tiled stride 3
    "tiled_open": dict(Lx=9, Ly=8, L_c=3, stride=3, schedule=P.SCHEDULE_TILED, periodic=0, T=0.1),
    # a chain split into segments
    "chain": dict(Lx=24, Ly=1, L_c=4, stride=4, schedule=P.SCHEDULE_TILED, periodic=1, T=0.1),
}


def _oracle_model(c):
    return oracle.Model(Lx=c["Lx"], Ly=c["Ly"], Lc=c["L_c"], JH=8.0, mu=-6.5, T=c["T"],
                        lattice_periodic=c["periodic"], schedule=c["schedule"], stride=c.get("stride", 0), seed=11)


def _config(c):
    return P.Config(**c, J_H=8.0, mu=-6.5, seed=11)


class OracleBackend:
    """The oracle behind the strip driver: the listed visits of a stage all
    read the configuration at the stage's start (Sec. II.c steps a-f per
    visit), then their decisions are written."""

    def __init__(self, m, S):
        self.m, self.S, self.rec = m, S.copy(), {}

    def run_visits(self, sites, sweep):
        S0 = self.S.copy()
        for v in (int(x) for x in sites):
            Fo = oracle.cluster_free_energy(self.m, S0, v)
            sn = oracle.propose(self.m, sweep, v, S0[v])
            Fn = oracle.cluster_free_energy(self.m, S0, v, sn)
            lnu = math.log(oracle.uniform2(self.m.seed, sweep, v, 2)[0])
            acc = lnu < -(Fn - Fo) / self.m.T
            if acc:
                self.S[v] = sn
            self.rec[(sweep, v)] = (Fo, Fn, lnu, acc)

    def gather(self, sites):
        return torch.from_numpy(self.S[np.asarray(sites, dtype=np.int64)].copy())

    def scatter(self, sites, spins):
        self.S[np.asarray(sites, dtype=np.int64)] = spins.numpy()


def test_plan_partitions_each_stage_and_reads_exactly_the_windows():
    for name, c in CASES.items():
        cfg, m = _config(c), _oracle_model(c)
        for world in (2, 3):
            if cfg.Ly > 1 and world * (2 if c["schedule"] == P.SCHEDULE_BLOCK else 1) > cfg.Ly:
                continue
            plan = strips.StripPlan.build(cfg, world)
            for s, stage in enumerate(plan.stages):
                parts = np.concatenate([plan.owned[r][s] for r in range(world)])
                assert sorted(parts.tolist()) == sorted(stage.tolist()), name
            for r in range(world):
                # the windows of rank r's visits, from the oracle's own window rule
                want = np.zeros(cfg.N, dtype=bool)
                for st in plan.owned[r]:
                    for v in st:
                        for g in range(cfg.N):
                            if oracle.in_window(m, int(v), g):
                                want[g] = True
                assert np.array_equal(plan.reads[r], want), (name, world, r)
                for s in range(plan.n_stages):
                    for q in range(world):
                        sent = plan.send[s][r][q]
                        assert np.all(np.isin(sent, plan.owned[r][s]))
                        if q != r:
                            assert np.all(plan.reads[q][sent])
                            rest = np.setdiff1d(plan.owned[r][s], sent)
                            assert not np.any(plan.reads[q][rest])


def test_halo_is_L_c_minus_one_rows_around_each_strip():
    # 16x16 torus, 4x4 clusters, central update site (o = 2), 2 ranks: rank
    # 0 owns rows 0..7 and reads rows 14, 15 (o below) and 0..8 (L_c-1-o above).
    cfg = P.Config(Lx=16, Ly=16, L_c=4, stride=4)
    plan = strips.StripPlan.build(cfg, 2)
    assert plan.strips == [[(0, 8)], [(8, 16)]] and plan.halo_rows() == 3
    rows = sorted(set((np.flatnonzero(plan.reads[0]) // 16).tolist()))
    assert rows == [0, 1, 2, 3, 4, 5, 6, 7, 8, 14, 15]
    assert len(rows) - 8 == plan.halo_rows()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _DroppingExchange(strips.TorchDistExchange):
    """An exchange that loses every message (the receiver keeps stale halo
    spins): the partitioned sweep must then differ from the sequential one."""

    def __call__(self, out, expected):
        got = super().__call__(out, expected)
        return {}


def _rank_main(rank, world, port, name, sweeps, out, drop=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASES[name]
        cfg, m = _config(c), _oracle_model(c)
        plan = strips.StripPlan.build(cfg, world)
        be = OracleBackend(m, oracle.init_spins(m))
        ex = _DroppingExchange("cpu") if drop else strips.TorchDistExchange("cpu")
        rk = strips.StripRank(plan, rank, be, ex)
        for sw in range(sweeps):
            rk.sweep(sw)
        mine = np.concatenate(plan.owned[rank][0:])  # every site this rank owns
        out[rank] = (mine, be.S[mine], be.rec)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", sorted(CASES))
def test_two_gloo_ranks_reproduce_the_sequential_oracle_sweep(name):
    world, sweeps = 2, 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, sweeps, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    m = _oracle_model(CASES[name])
    S = oracle.init_spins(m)
    recs = []
    for sw in range(sweeps):
        S, rec = oracle.sweep(m, S, sw)
        recs.append(rec)
    seen = 0
    for r in range(world):
        mine, spins, rec = out[r]
        assert np.array_equal(spins, S[mine])  # bit for bit
        for sw in range(sweeps):
            for k, v in enumerate(recs[sw].site):
                if (sw, int(v)) in rec:
                    Fo, Fn, lnu, acc = rec[(sw, int(v))]
                    assert (Fo, Fn, lnu) == (recs[sw].F_old[k], recs[sw].F_new[k], recs[sw].lnu[k])
                    assert acc == bool(recs[sw].accepted[k])
                    seen += 1
    assert seen == sweeps * m.N  # every visit ran on exactly one rank


def test_without_the_halo_exchange_the_strips_diverge():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, "tiled_periodic", 2, out, True)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    m = _oracle_model(CASES["tiled_periodic"])
    S = oracle.init_spins(m)
    for sw in range(2):
        S, _ = oracle.sweep(m, S, sw)
    assert any(not np.array_equal(out[r][1], S[out[r][0]]) for r in range(2))

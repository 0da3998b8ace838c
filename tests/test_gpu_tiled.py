"""The register-tiled FP32 Householder pass (launch configuration reduction
= PTCA_REDUCTION_TILED, 4-warp CTAs, orders up to 128).

It stores the cluster matrix as 4x4 tiles and reorganises the fused
update + product pass of the reduction (Sec. II.c step b); the arithmetic
per element is that of the row-chunked pass.  Checked against the oracle's
solves (free energies, ln u, decisions, spins), against the FP64 path on
the free-energy-difference scale, and against the row-chunked pass (same
decisions and spins, free energies to rounding), on orders that fill the
tiles exactly (32, 64, 128) and ragged ones (n mod 4 = 2, clipped windows of
open lattices, chains down to n = 4)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests.test_gpu_parity import _check_sweep_against_oracle
from tests.test_gpu_precision import MIXED_DF_BOUND, _level_scale

pytestmark = pytest.mark.gpu

TILED_STAGES = (P.PIPELINE_STAGES, 4, 0, P.REDUCTION_TILED)
TILED_OVERLAP = (P.PIPELINE_OVERLAP, 4, 0, P.REDUCTION_TILED)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


@pytest.mark.parametrize("lat", [
    dict(Lx=8, Ly=8, L_c=4),                                   # n = 32, every tile full
    dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6),           # n = 18 .. 72, clipped, n mod 4 = 2 included
    dict(Lx=24, Ly=1, L_c=2, stride=2),                        # chain, n = 4: one block
    dict(Lx=30, Ly=1, L_c=5, stride=5),                        # chain, n = 10: a padded second block
])
def test_tiled_reduction_against_the_oracle_every_visit(lat):
    cfg = P.Config(**lat, t=1.0, J_H=8.0, mu=-6.5, T=0.05, seed=3, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, launch=TILED_STAGES)


def test_tiled_reduction_against_the_oracle_n128_overlap():
    # 24x24 torus, 8x8 clusters (n = 128, 32 tile rows), the paper's block
    # schedule, cone proposals: sampled visits plus those nearest the
    # Metropolis threshold (re-solved), through the overlapped pipeline.
    cfg = P.Config(Lx=24, Ly=24, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                   T=0.05, mu=-6.5, seed=9, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=12, near=6, launch=TILED_OVERLAP)


@pytest.mark.parametrize("lat", [dict(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK),
                                 dict(Lx=23, Ly=21, L_c=7, periodic=0, stride=7)])
def test_tiled_and_row_chunked_passes_compute_the_same_chain(lat):
    cfg = P.Config(**lat, proposal=P.PROPOSAL_CONE, T=0.05, mu=-6.5, seed=17, precision=P.MIXED)
    runs = []
    for launch in [(P.PIPELINE_STAGES, 4, 0, P.REDUCTION_ROWS), TILED_STAGES, TILED_OVERLAP]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, *launch)
        got = P.ptca_get_launch_config(ctx.h)
        assert (got.pipeline, got.warps_per_cta, got.ctas_per_sm, got.reduction) == launch
        ctx.sweep(2)
        rec = [x.cpu().numpy() for x in ctx.record()]
        runs.append((ctx.spins().cpu().numpy(), rec))
        ctx.close()
    S_ref, (site, Fo, Fn, lnu, acc) = runs[0]
    for S, (site2, Fo2, Fn2, lnu2, acc2) in runs[1:]:
        assert np.array_equal(site, site2) and np.array_equal(acc, acc2)
        assert np.array_equal(lnu, lnu2)
        assert np.array_equal(S, S_ref)
        assert np.max(np.abs(Fo2 - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5
        assert np.max(np.abs(Fn2 - Fn) / np.maximum(1.0, np.abs(Fn))) < 1e-5
    # the two tiled pipelines run the same kernel on the same snapshots: bit for bit
    for x, y in zip(runs[1][1], runs[2][1]):
        assert np.array_equal(x, y)


def test_tiled_dF_error_on_the_free_energy_difference_scale():
    # Stage 0 of the 100x100 headline, unguarded (margin 0): sampled visits'
    # dF against the oracle's, on the scale max(|dF|, sum_k |eps_k - mu| f_k / n).
    base = dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                T=0.05, mu=-6.5, seed=0)
    m = oracle.Model(Lx=100, Ly=100, Lc=8, JH=8.0, mu=-6.5, T=0.05, schedule=oracle.SCHEDULE_BLOCK,
                     proposal=oracle.PROPOSAL_CONE, cone_deg=30.0, seed=0)
    cfg = P.Config(**base, precision=P.MIXED)
    stage0 = P.ptca_schedule(cfg)[0]
    ctx = P.Context(cfg)
    P.ptca_set_launch_config(ctx.h, *TILED_STAGES)
    P.ptca_set_resolve_margin(ctx.h, 0.0)
    ctx.sweep(1)
    site, Fo, Fn, _, _ = (x.cpu().numpy() for x in ctx.record())
    ctx.close()
    S0 = oracle.init_spins(m)
    worst = 0.0
    for k in range(0, len(stage0), len(stage0) // 12)[:12]:
        s = int(stage0[k])
        assert site[k] == s
        sn = oracle.propose(m, 0, s, S0[s])
        e_old = oracle.eigvalsh(oracle.cluster_hamiltonian(m, S0, s)[0])
        dF = oracle.cluster_free_energy(m, S0, s, sn) - oracle.free_energy(e_old, m.mu, m.T)
        scale = max(abs(dF), _level_scale(e_old, m.mu, m.T))
        worst = max(worst, abs((Fn[k] - Fo[k]) - dF) / scale)
    assert worst <= MIXED_DF_BOUND, worst


def test_tiled_reduction_configuration_is_validated():
    mixed = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.MIXED))
    for bad in [(P.PIPELINE_STAGES, 8, 0, P.REDUCTION_TILED),       # 8-warp CTAs
                (P.PIPELINE_PERSISTENT, 4, 0, P.REDUCTION_TILED),   # persistent kernel
                (P.PIPELINE_GRAPH, 4, 0, P.REDUCTION_TILED)]:
        with pytest.raises(P.PtcaError):
            P.ptca_set_launch_config(mixed.h, *bad)
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(mixed.h, P.PIPELINE_STAGES, 4, 0, 3)  # no such reduction
    got = P.ptca_get_launch_config(mixed.h)
    assert got.reduction == P.REDUCTION_ROWS  # unchanged by the rejected calls
    mixed.close()
    fp64 = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.FP64))
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(fp64.h, *TILED_STAGES)
    fp64.close()
    big = P.Context(P.Config(Lx=20, Ly=20, L_c=10, precision=P.MIXED))  # n = 200 > 128
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(big.h, *TILED_STAGES)
    big.close()


def test_autotune_offers_the_tiled_reduction():
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=23,
                   precision=P.MIXED)
    ctx = P.Context(cfg)
    best, table = P.ptca_autotune(ctx.h, 1)
    tiled = [c for c in table["candidates"] if c["reduction"] == 1]
    assert {c["pipeline"] for c in tiled} == {"stages", "overlap"}
    assert all(c["warps_per_cta"] == 4 and c["ms_per_sweep"] is not None for c in tiled)
    assert table["best"]["reduction"] == P.ptca_get_launch_config(ctx.h).reduction == best.reduction
    ctx.close()

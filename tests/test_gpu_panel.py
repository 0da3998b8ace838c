"""The blocked (panel) FP32 Householder reduction (launch configuration
panel_width = 2, 4 or 8, 8-warp CTAs, orders up to 128): panels of b
reflectors, each formed from the panel-start matrix with the panel's earlier
pairs as corrections, and one rank-2b update of the trailing block per panel
(Sec. II.c step b).

Checked against the oracle's solves (free energies, ln u, decisions, spins)
on orders 4 ... 128 including ragged clipped windows and panels cut short at
the end of the reduction, against the FP64 path on the free-energy-difference
scale, and against the unblocked reduction (same decisions and spins, free
energies to rounding)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests.test_gpu_parity import _check_sweep_against_oracle
from tests.test_gpu_precision import MIXED_DF_BOUND, _level_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _panel(b, pipeline=P.PIPELINE_STAGES):
    return (pipeline, 8, 0, P.REDUCTION_ROWS, b)


@pytest.mark.parametrize("b", [2, 4, 8])
@pytest.mark.parametrize("lat", [
    dict(Lx=8, Ly=8, L_c=4),                                   # n = 32
    dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6),           # n = 18 .. 72, clipped
    dict(Lx=24, Ly=1, L_c=2, stride=2),                        # chain, n = 4: one short panel
    dict(Lx=30, Ly=1, L_c=5, stride=5),                        # chain, n = 10
])
def test_panel_reduction_against_the_oracle_every_visit(b, lat):
    cfg = P.Config(**lat, t=1.0, J_H=8.0, mu=-6.5, T=0.05, seed=3, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, launch=_panel(b))


@pytest.mark.parametrize("b", [2, 8])
def test_panel_reduction_against_the_oracle_n128_overlap(b):
    cfg = P.Config(Lx=24, Ly=24, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                   T=0.05, mu=-6.5, seed=9, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=12, near=6, launch=_panel(b, P.PIPELINE_OVERLAP))


def test_panel_and_unblocked_reductions_compute_the_same_chain():
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, mu=-6.5,
                   seed=17, precision=P.MIXED)
    runs = []
    for launch in [(P.PIPELINE_STAGES, 8, 0, 0, 0), _panel(2), _panel(4), _panel(8),
                   _panel(8, P.PIPELINE_OVERLAP)]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, *launch)
        got = P.ptca_get_launch_config(ctx.h)
        assert (got.pipeline, got.warps_per_cta, got.ctas_per_sm, got.reduction, got.panel_width) == launch
        ctx.sweep(2)
        runs.append((ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    S_ref, (site, Fo, Fn, lnu, acc) = runs[0]
    for S, (site2, Fo2, Fn2, lnu2, acc2) in runs[1:]:
        assert np.array_equal(site, site2) and np.array_equal(acc, acc2) and np.array_equal(lnu, lnu2)
        assert np.array_equal(S, S_ref)
        assert np.max(np.abs(Fo2 - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5
        assert np.max(np.abs(Fn2 - Fn) / np.maximum(1.0, np.abs(Fn))) < 1e-5
    for x, y in zip(runs[3][1], runs[4][1]):  # same kernel, two pipelines: bit for bit
        assert np.array_equal(x, y)


@pytest.mark.parametrize("b", [2, 8])
def test_panel_dF_error_on_the_free_energy_difference_scale(b):
    base = dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                T=0.05, mu=-6.5, seed=0)
    m = oracle.Model(Lx=100, Ly=100, Lc=8, JH=8.0, mu=-6.5, T=0.05, schedule=oracle.SCHEDULE_BLOCK,
                     proposal=oracle.PROPOSAL_CONE, cone_deg=30.0, seed=0)
    cfg = P.Config(**base, precision=P.MIXED)
    stage0 = P.ptca_schedule(cfg)[0]
    ctx = P.Context(cfg)
    P.ptca_set_launch_config(ctx.h, *_panel(b))
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


def test_panel_configuration_is_validated_and_autotuned():
    ctx = P.Context(P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, T=0.05, seed=23, precision=P.MIXED))
    for bad in [(P.PIPELINE_STAGES, 4, 0, 0, 4),                # 4-warp CTAs
                (P.PIPELINE_PERSISTENT, 8, 0, 0, 4),            # persistent kernel
                (P.PIPELINE_STAGES, 8, 0, P.REDUCTION_TILED, 4)]:
        with pytest.raises(P.PtcaError):
            P.ptca_set_launch_config(ctx.h, *bad)
    for bad_b in (3, 16, -1):
        with pytest.raises(P.PtcaError):
            P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 8, 0, 0, bad_b)
    assert P.ptca_get_launch_config(ctx.h).panel_width == 0
    best, table = P.ptca_autotune(ctx.h, 1)
    panels = [c for c in table["candidates"] if c["panel_width"] > 1]
    assert {c["panel_width"] for c in panels} == {2, 4, 8}
    assert all(c["warps_per_cta"] == 8 and c["ms_per_sweep"] is not None for c in panels)
    assert table["best"]["panel_width"] == P.ptca_get_launch_config(ctx.h).panel_width == best.panel_width
    ctx.close()
    fp64 = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.FP64))
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(fp64.h, *_panel(4))
    fp64.close()

"""Large traveling clusters (the paper's N_c = 12^2 and 16^2, Sec. VII.a):
matrix orders above the shared-memory kernels' (242, 288, 512) run on the
global-memory Householder path with 16-warp CTAs.  Sweeps against the oracle
visit by visit in FP64 and mixed precision, and bit identity of the
per-stage and overlapped pipelines with every decision re-solved."""
import numpy as np
import pytest
import torch

import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests.test_gpu_parity import _check_sweep_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


@pytest.mark.parametrize("prec,width", [(P.FP64, 16), (P.MIXED, 16), (P.MIXED, 8)])
@pytest.mark.parametrize("Lc", [11, 12])
def test_large_cluster_sweeps_match_oracle(prec, width, Lc):
    # width 16: one CTA per matrix, the matrix in global memory; width 8
    # (PTCA_MIXED): a thread-block cluster per matrix, the matrix in
    # distributed shared memory.
    cfg = P.Config(Lx=2 * Lc, Ly=2 * Lc, L_c=Lc, schedule=P.SCHEDULE_BLOCK, J_H=8.0, mu=-6.5, T=0.1, seed=Lc,
                   precision=prec, proposal=P.PROPOSAL_CONE)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=4, launch=(P.PIPELINE_STAGES, width))


@pytest.mark.parametrize("width", [16, 8])
def test_16x16_clusters_n512_match_oracle(width):
    cfg = P.Config(Lx=32, Ly=32, L_c=16, schedule=P.SCHEDULE_BLOCK, J_H=8.0, mu=-6.5, T=0.1, seed=16,
                   precision=P.MIXED, proposal=P.PROPOSAL_CONE)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=2, launch=(P.PIPELINE_STAGES, width))


@pytest.mark.parametrize("width", [16, 8])
@pytest.mark.parametrize("margin", [None, 1e6])
def test_large_cluster_pipelines_are_bit_identical(margin, width):
    # Default margin: most decisions come from the FP32 solves of the
    # concurrent independent and dependent launches; 1e6: every decision is
    # re-solved in double-float.
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, T=0.1, seed=3, precision=P.MIXED,
                   proposal=P.PROPOSAL_CONE)
    runs = []
    for pl in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP, P.PIPELINE_OVERLAP):
        ctx = P.Context(cfg)
        if margin is not None:
            P.ptca_set_resolve_margin(ctx.h, margin)
        P.ptca_set_launch_config(ctx.h, pl, width, 0)
        st = ctx.sweep(2)
        if margin is not None:
            assert st.resolved == 2 * cfg.N
        runs.append((ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    for S, rec in runs[1:]:
        assert np.array_equal(runs[0][0], S)
        for a, b in zip(runs[0][1], rec):
            assert np.array_equal(a, b)


def test_large_cluster_limits_are_reported():
    ctx = P.Context(P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED))
    for pl in (P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH):
        with pytest.raises(P.PtcaError) as e:
            P.ptca_set_launch_config(ctx.h, pl, 8, 0)
        assert e.value.status in (1, 6)
    with pytest.raises(P.PtcaError) as e:
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 4, 0)
    assert e.value.status == 6
    assert P.ptca_get_launch_config(ctx.h).warps_per_cta == 16
    with pytest.raises(P.PtcaError) as e:
        P.ptca_set_checker(ctx.h, True)
    assert e.value.status == 6
    best, table = P.ptca_autotune(ctx.h, 1)
    assert best.pipeline in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP)
    ctx.close()

"""PTCA_MIXED decision guard (FP32 reduction, FP64 eigenvalues and dF, FP64
re-solve of decisions within the margin).

With the guard, a mixed-precision sweep must take exactly the decisions of
the FP64 path wherever the FP64 margin |ln u + dF/T| exceeds 1e-6; since
every decision of a stage then agrees, the spins entering the next stage
agree too and whole sweeps coincide."""
import numpy as np
import pytest
import torch

import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _one_sweep(cfg, pipeline, margin=None):
    ctx = P.Context(cfg)
    P.ptca_set_pipeline(ctx.h, pipeline)
    if margin is not None:
        P.ptca_set_resolve_margin(ctx.h, margin)
    st = ctx.sweep(1)
    rec = [x.cpu().numpy() for x in ctx.record()]
    S = ctx.spins().cpu().numpy()
    ctx.close()
    return st, rec, S


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("pipeline", [P.PIPELINE_STAGES, P.PIPELINE_GRAPH])
def test_guarded_mixed_sweep_takes_the_fp64_decisions(seed, pipeline):
    base = dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                T=0.05, mu=-6.5, seed=seed)
    st64, r64, S64 = _one_sweep(P.Config(**base, precision=P.FP64), pipeline)
    st32, r32, S32 = _one_sweep(P.Config(**base, precision=P.MIXED), pipeline)
    site64, Fo64, Fn64, lnu, acc64 = r64
    site32, Fo32, Fn32, lnu32, acc32 = r32
    assert np.array_equal(site64, site32)
    margin = np.abs(lnu + (Fn64 - Fo64) / base["T"])
    assert np.all(margin > 1e-6)
    assert np.array_equal(acc64, acc32)
    assert np.max(np.abs(S64 - S32)) < 1e-13
    assert st32.resolved > 0  # the guard did fire on this workload
    assert st32.resolved < 0.05 * st32.attempts
    # Deferred visits carry FP64 free energies; the rest are within the mixed tolerance.
    assert np.max(np.abs(Fo32 - Fo64) / np.abs(Fo64)) < 1e-5


def test_guard_off_resolves_nothing_and_fp64_rejects_guard():
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=3,
                   precision=P.MIXED)
    st, _, _ = _one_sweep(cfg, P.PIPELINE_GRAPH, margin=0.0)
    assert st.resolved == 0
    st, _, _ = _one_sweep(cfg, P.PIPELINE_GRAPH, margin=1.0)
    assert st.resolved > 0
    ctx = P.Context(P.Config(Lx=8, Ly=8, L_c=4, precision=P.FP64))
    with pytest.raises(P.PtcaError):
        P.ptca_set_resolve_margin(ctx.h, 1e-2)
    ctx.close()

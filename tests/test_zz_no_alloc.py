"""ptca_sweep_noalloc: the sweep for callers that cannot allocate device
memory (their own pool owns the device, or allocation in their loop is not
acceptable).  It must give the same per-visit free energies, decisions and
spins as the context-based ptca_sweep, call after call, while keeping its
working memory in the library's fixed device array -- in PTCA_MIXED with the
same re-solve of near-threshold decisions, so that its decisions equal the
FP64 path's.

This file is named to be collected last."""
import numpy as np
import pytest
import torch

import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build

pytestmark = pytest.mark.gpu

TOL = {P.FP64: 1e-9, P.MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.lib()


def _noalloc(cfg, spins, sweep):
    N = cfg.N
    F_out = torch.full((2 * N,), float("nan"), dtype=torch.float64, device="cuda")
    acc_out = torch.full((N,), 7, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    P.ptca_sweep_noalloc(cfg, spins, sweep, F_out, acc_out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return F_out, acc_out


@pytest.mark.parametrize("cfg", [
    P.Config(Lx=8, Ly=8, L_c=4, T=0.05, mu=-6.5, seed=0, precision=P.FP64, schedule=P.SCHEDULE_BLOCK),
    P.Config(Lx=10, Ly=10, L_c=8, stride=5, T=0.05, mu=-6.5, seed=3, precision=P.MIXED,
             proposal=P.PROPOSAL_CONE, cone_deg=30.0),
    P.Config(Lx=8, Ly=8, L_c=4, T=0.1, mu=4.0, U=8.0, m_step=0.5, seed=5, precision=P.FP64,
             model=P.MODEL_HUBBARD_MF, schedule=P.SCHEDULE_BLOCK),
    P.Config(Lx=64, Ly=1, L_c=8, T=0.1, mu=0.0, lam=1.5, K=1.0, m_step=0.4, seed=6, precision=P.MIXED,
             model=P.MODEL_HOLSTEIN, schedule=P.SCHEDULE_TILED, stride=8, update_offset=4),
    P.Config(Lx=6, Ly=6, Lz=6, L_c=3, stride=3, T=0.1, mu=-6.5, seed=7, precision=P.FP64),
])
def test_noalloc_sweeps_match_context_sweeps(cfg):
    N = cfg.N
    ctx = P.Context(cfg)
    spins = ctx.spins().clone()
    tol = TOL[cfg.precision]
    for sweep in range(2):  # two calls in a row share the library's array
        ctx.sweep(1)
        _, Fo, Fn, _, acc = ctx.record()
        F_out, acc_out = _noalloc(cfg, spins, sweep)
        scale = torch.clamp(Fo.abs(), min=1.0)
        assert torch.max((F_out[:N] - Fo).abs() / scale).item() <= tol
        assert torch.max((F_out[N:] - Fn).abs() / scale).item() <= tol
        assert torch.equal(acc_out, acc)
        assert torch.max((spins - ctx.spins()).abs()).item() <= 1e-12
    ctx.close()


def test_noalloc_mixed_guard_matches_fp64_decisions_at_full_size():
    # The 100x100 torus with 8x8 clusters (n = 128), 30-degree cone proposals,
    # T = 0.05: about 1 % of the visits fall within the re-solve band.  The
    # mixed context sweep re-solves them (resolved > 0); the no-allocation
    # sweep must re-solve the same visits and so decide every visit as the
    # plain FP64 path does, two calls in a row.
    base = dict(Lx=100, Ly=100, L_c=8, T=0.05, mu=-6.5, seed=0, schedule=P.SCHEDULE_BLOCK,
                proposal=P.PROPOSAL_CONE, cone_deg=30.0)
    cfg = P.Config(**base, precision=P.MIXED)
    ctx = P.Context(cfg)
    ctx64 = P.Context(P.Config(**base, precision=P.FP64))
    spins = ctx.spins().clone()
    N = cfg.N
    for sweep in range(2):
        st = ctx.sweep(1)
        assert st.resolved > 0
        _, Fo, Fn, _, acc = ctx.record()
        ctx64.sweep(1)
        _, Fo64, Fn64, _, acc64 = ctx64.record()
        F_out, acc_out = _noalloc(cfg, spins, sweep)
        assert torch.equal(acc_out, acc)
        assert torch.equal(acc_out, acc64)
        scale = torch.clamp(Fo64.abs(), min=1.0)
        assert torch.max((F_out[:N] - Fo).abs() / scale).item() <= TOL[P.MIXED]
        assert torch.max((F_out[N:] - Fn).abs() / scale).item() <= TOL[P.MIXED]
        assert torch.equal(spins, ctx64.spins())
    ctx.close()
    ctx64.close()


def test_noalloc_rejects_what_its_array_or_shared_memory_cannot_hold():
    # 10x10 clusters (n = 200) in PTCA_MIXED: the re-solve matrix does not
    # fit in shared memory, and the call refuses rather than run unguarded.
    cfg = P.Config(Lx=20, Ly=20, L_c=10, stride=10, precision=P.MIXED)
    spins = torch.zeros((cfg.N, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PtcaError) as e:
        P.ptca_sweep_noalloc(cfg, spins, 0)
    assert e.value.status == 6 and "re-solve" in str(e.value)
    cfg = P.Config(Lx=200, Ly=200, L_c=4)
    with pytest.raises(P.PtcaError) as e:
        P.ptca_sweep_noalloc(cfg, torch.zeros((cfg.N, 3), dtype=torch.float64, device="cuda"), 0)
    assert e.value.status == 1 and "at most 16384" in str(e.value)

"""ptca_sweep_noalloc: the sweep for callers that cannot allocate device
memory (their own pool owns the device, or allocation in their loop is not
acceptable).  It must give the same per-visit free energies, decisions and
spins as the context-based ptca_sweep, call after call, while keeping its
working memory in the library's fixed device array.

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
    stages = P.ptca_schedule(cfg)
    stage_start = np.concatenate([[0], np.cumsum([len(s) for s in stages])]).astype(np.int32)
    sites = torch.from_numpy(np.concatenate(stages).astype(np.int32)).cuda()
    N = cfg.N
    ctx = P.Context(cfg)
    spins = ctx.spins().clone()
    tol = TOL[cfg.precision]
    for sweep in range(2):  # two calls in a row share the library's array
        ctx.sweep(1)
        _, Fo, Fn, _, acc = ctx.record()
        F_out = torch.full((2 * N,), float("nan"), dtype=torch.float64, device="cuda")
        acc_out = torch.full((N,), 7, dtype=torch.uint8, device="cuda")
        P.ptca_sweep_noalloc(cfg, sites, stage_start, spins, sweep, F_out, acc_out)
        torch.cuda.synchronize()
        scale = torch.clamp(Fo.abs(), min=1.0)
        assert torch.max((F_out[:N] - Fo).abs() / scale).item() <= tol
        assert torch.max((F_out[N:] - Fn).abs() / scale).item() <= tol
        assert torch.equal(acc_out, acc)
        assert torch.max((spins - ctx.spins()).abs()).item() <= 1e-12
    ctx.close()


def test_noalloc_rejects_lattices_beyond_its_array():
    cfg = P.Config(Lx=200, Ly=200, L_c=4)
    stages = P.ptca_schedule(cfg)
    stage_start = np.concatenate([[0], np.cumsum([len(s) for s in stages])]).astype(np.int32)
    sites = torch.zeros(1, dtype=torch.int32, device="cuda")
    spins = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PtcaError) as e:
        P.ptca_sweep_noalloc(cfg, sites, stage_start, spins, 0)
    assert e.value.status == 1 and "at most 16384" in str(e.value)

"""The strip decomposition on the GPU path, two ranks emulated in one
process on one GPU: two contexts hold the two ranks' copies of the
configuration, each runs the visits of its strips through ptca_stage_run,
and after every stage the halo spins move between them through
ptca_get_sites / ptca_set_sites (the messages the ranks would exchange).  No
kernel waits on another: the ranks' launches alternate on one stream.  The
union of the strips must equal a single-context ptca_sweep bit for bit, in
FP64 and in guarded mixed precision (paper Sec. III.b, Fig. 4)."""
import numpy as np
import pytest
import torch

import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build, strips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    P.lib()


def _emulated(cfg, world, sweeps):
    plan = strips.StripPlan.build(cfg, world)
    ctxs = [P.Context(cfg) for _ in range(world)]
    ranks = [strips.StripRank(plan, r, strips.GpuStripBackend(ctxs[r]), None) for r in range(world)]
    for sw in range(sweeps):
        for s in range(plan.n_stages):
            outs = [rk.run_stage(s, sw) for rk in ranks]
            for r, rk in enumerate(ranks):
                rk.finish_stage(s, {q: outs[q][r] for q in range(world) if r in outs[q]})
    spins = [c.spins() for c in ctxs]
    out = torch.empty_like(spins[0])
    for r in range(world):
        mine = torch.from_numpy(np.concatenate(plan.owned[r]).astype(np.int64)).cuda()
        out[mine] = spins[r][mine]
    for c in ctxs:
        c.close()
    return out


@pytest.mark.parametrize("case", [
    dict(Lx=32, Ly=32, L_c=8, stride=8, precision=P.FP64, proposal=P.PROPOSAL_SPHERE, T=0.05),
    dict(Lx=32, Ly=32, L_c=8, stride=8, precision=P.MIXED, proposal=P.PROPOSAL_SPHERE, T=0.05),
    dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED, proposal=P.PROPOSAL_CONE,
         cone_deg=30.0, T=0.05),
    dict(Lx=40, Ly=40, L_c=10, stride=10, periodic=0, J_H=6.0, mu=-4.5, T=0.1, precision=P.MIXED),
])
def test_emulated_strips_equal_the_single_domain_sweep(case):
    cfg = P.Config(**{"mu": -6.5, "seed": 3, **case})
    world = 2 if cfg.schedule == P.SCHEDULE_BLOCK else 3
    sweeps = 2
    got = _emulated(cfg, world, sweeps)
    ref = P.Context(cfg)
    P.ptca_set_pipeline(ref.h, P.PIPELINE_STAGES)
    ref.sweep(sweeps)
    want = ref.spins()
    ref.close()
    assert torch.equal(got, want)


def test_stage_run_validates_its_site_list():
    cfg = P.Config(Lx=16, Ly=16, L_c=4, stride=4)
    ctx = P.Context(cfg)
    stages = P.ptca_schedule(cfg)
    for bad in ([0, 0], [-1], [cfg.N], np.concatenate([stages[0][:1], stages[1][:1]])):
        with pytest.raises(P.PtcaError) as e:
            P.ptca_stage_run(ctx.h, 0, np.asarray(bad, dtype=np.int32))
        assert e.value.status == 1
    ctx.close()

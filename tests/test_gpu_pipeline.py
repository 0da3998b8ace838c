"""Stage pipeline (persistent launch, device-wide barrier, CUDA graph,
overlapped re-solve) and ragged window sizes.

The four launch modes must give bit-identical sweeps: they run the same
per-cluster code on the same stage snapshots with the same counter-based
random numbers.  The bounded barrier must give up and report a timeout
instead of hanging.  Open lattices with L_c = 10 give windows from 5x5 to
10x10 (n = 50 ... 200), processed largest first."""
import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests import inputs
from tests.test_gpu_parity import _check_sweep_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
@pytest.mark.parametrize("lat", [dict(Lx=16, Ly=16, L_c=4, schedule=P.SCHEDULE_BLOCK),
                                 dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6)])
def test_pipelines_give_identical_sweeps(prec, lat):
    cfg = P.Config(**lat, T=0.1, mu=-6.5, seed=5, precision=prec, proposal=P.PROPOSAL_CONE)
    runs = {}
    for mode in (P.PIPELINE_STAGES, P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH, P.PIPELINE_OVERLAP):
        ctx = P.Context(cfg)
        P.ptca_set_pipeline(ctx.h, mode)
        recs = []
        for _ in range(3):  # three single-sweep calls: the RNG sweep counter must advance
            st = ctx.sweep(1)
            assert st.attempts == cfg.N and st.eigensolves == 2 * cfg.N
            recs.append([x.cpu().numpy() for x in ctx.record()])
        st = ctx.sweep(2)  # one two-sweep call
        recs.append([x.cpu().numpy() for x in ctx.record()])
        runs[mode] = (ctx.spins().cpu().numpy(), recs)
        ctx.close()
    S0, r0 = runs[P.PIPELINE_STAGES]
    for mode in (P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH, P.PIPELINE_OVERLAP):
        S, r = runs[mode]
        assert np.array_equal(S, S0)
        for a, b in zip(r, r0):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_barrier_timeout_is_reported_and_gpu_stays_usable():
    status = P.ptca_selftest_barrier_timeout(4, 0.2)
    assert status == 4  # PTCA_ERR_TIMEOUT
    cfg = P.Config(Lx=8, Ly=8, L_c=4, seed=1)
    ctx = P.Context(cfg)
    st = ctx.sweep(1)
    assert st.attempts == 64
    ctx.close()


def test_sweep_rejects_unknown_pipeline():
    ctx = P.Context(P.Config(Lx=8, Ly=8, L_c=4))
    with pytest.raises(P.PtcaError):
        P.ptca_set_pipeline(ctx.h, 7)
    ctx.close()


@pytest.mark.parametrize("prec", [P.MIXED])
def test_open_lattice_L10_ragged_windows_up_to_n200(prec):
    # Open lattice, L_c = 10 (windows 5x5 ... 10x10, n = 50 ... 200), J_H = 6,
    # mu = -4.5, T = 0.1: the uneven-batch workload at reduced lattice size.
    cfg = P.Config(Lx=24, Ly=22, L_c=10, periodic=0, stride=10, J_H=6.0, mu=-4.5, T=0.1, seed=7, precision=prec)
    stages = P.ptca_schedule(cfg)
    sizes = set()
    m = oracle.Model(Lx=cfg.Lx, Ly=cfg.Ly, Lc=10, lattice_periodic=0)
    for s in np.concatenate(stages)[::7]:
        _, (ex, ey) = oracle.cluster_hamiltonian(m, np.tile([0, 0, 1.0], (cfg.N, 1)), int(s))
        sizes.add(2 * ex * ey)
    assert max(sizes) == 200 and min(sizes) <= 72
    _check_sweep_against_oracle(cfg, sweeps=1, sample=5)


@pytest.mark.parametrize("lat", [(32, 8), (8, 4)])
def test_launch_configurations_compute_the_same_chain(lat):
    # CTA width (8 or 4 warps), pipeline and persistent CTAs per SM change
    # only how the work is laid out: with the decision guard the decisions,
    # hence the spins, are identical; free energies agree to rounding.
    L, Lc = lat
    cfg = P.Config(Lx=L, Ly=L, L_c=Lc, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=17,
                   precision=P.MIXED)
    runs = []
    for pl, nw, cps in [(P.PIPELINE_GRAPH, 8, 0), (P.PIPELINE_STAGES, 4, 0), (P.PIPELINE_PERSISTENT, 4, 0),
                        (P.PIPELINE_GRAPH, 4, 1), (P.PIPELINE_PERSISTENT, 8, 1), (P.PIPELINE_OVERLAP, 4, 0),
                        (P.PIPELINE_OVERLAP, 8, 0)]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, pl, nw, cps)
        got = P.ptca_get_launch_config(ctx.h)
        assert (got.pipeline, got.warps_per_cta, got.ctas_per_sm) == (pl, nw, cps)
        ctx.sweep(2)
        rec = [x.cpu().numpy() for x in ctx.record()]
        runs.append((ctx.spins().cpu().numpy(), rec))
        ctx.close()
    S_ref, (site, Fo, Fn, lnu, acc) = runs[0]
    for S, (site2, Fo2, Fn2, lnu2, acc2) in runs[1:]:
        assert np.array_equal(site, site2) and np.array_equal(acc, acc2)
        assert np.array_equal(S, S_ref)
        assert np.max(np.abs(Fo2 - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5


def test_autotune_restores_the_chain_and_applies_the_fastest():
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=23,
                   precision=P.MIXED)
    ctx = P.Context(cfg)
    ctx.sweep(1)
    S0 = ctx.spins().cpu().numpy()
    best, table = P.ptca_autotune(ctx.h, 2)
    assert np.array_equal(ctx.spins().cpu().numpy(), S0)
    got = P.ptca_get_launch_config(ctx.h)
    assert (got.pipeline, got.warps_per_cta, got.ctas_per_sm) == (best.pipeline, best.warps_per_cta, best.ctas_per_sm)
    timed = [c for c in table["candidates"] if c["ms_per_sweep"] is not None]
    assert len(timed) >= 6 and {c["warps_per_cta"] for c in timed} == {4, 8}
    fastest = min(timed, key=lambda c: c["ms_per_sweep"])
    names = {P.PIPELINE_STAGES: "stages", P.PIPELINE_PERSISTENT: "persistent", P.PIPELINE_GRAPH: "graph",
             P.PIPELINE_OVERLAP: "overlap"}
    assert {c["pipeline"] for c in timed} == set(names.values())
    assert (names[best.pipeline], best.warps_per_cta, best.ctas_per_sm) == (
        fastest["pipeline"], fastest["warps_per_cta"], fastest["ctas_per_sm"])
    # The next sweep continues the chain exactly as without the tuning.
    ctx.sweep(1)
    ref = P.Context(cfg)
    ref.sweep(2)
    assert np.array_equal(ctx.spins().cpu().numpy(), ref.spins().cpu().numpy())
    ctx.close()
    ref.close()


def test_launch_configuration_is_validated():
    ctx = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.FP64))
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_GRAPH, 4, 0)   # 4-warp kernels are FP32 only
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_GRAPH, 6, 0)
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_GRAPH, 8, 99)
    ctx.close()
    ctx = P.Context(P.Config(Lx=40, Ly=40, L_c=10, periodic=0, stride=10, precision=P.MIXED))  # n up to 200
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 4, 0)
    ctx.close()


def test_kernel_timing_counts_the_stage_launches():
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, T=0.05, seed=3, precision=P.MIXED)
    ctx = P.Context(cfg)
    ns = len(P.ptca_schedule(cfg))
    P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 8, 0)
    P.ptca_set_kernel_timing(ctx.h, True)
    ctx.sweep(2)
    kt = P.ptca_kernel_times(ctx.h)
    st_ms, st_n, rs_ms, rs_n = kt[:4]
    assert st_n == 2 * ns and rs_n == 2 * ns and st_ms > 0 and rs_ms >= 0
    assert kt.stage_matrices == 2 * 2 * cfg.N and kt.dependent_launches == 0
    # one stream: the stage launches do not overlap, their union is their sum
    assert abs(kt.stage_union_ms - st_ms) <= 1e-3 * st_ms + 0.05
    assert tuple(P.ptca_kernel_times(ctx.h)) == (0.0, 0, 0.0, 0, 0.0, 0, 0, 0, 0.0)   # read clears
    # Overlapped pipeline: the independent and the dependent visits of each
    # stage are separate launches; together they solve every matrix once.
    P.ptca_set_launch_config(ctx.h, P.PIPELINE_OVERLAP, 8, 0)
    ctx.sweep(2)
    kt = P.ptca_kernel_times(ctx.h)
    split = P.ptca_stage_split(cfg)
    assert kt.stage_launches == 2 * sum(1 for _, n in split if n > 0)
    assert kt.dependent_launches == 2 * sum(1 for o, n in split if o.size > n)
    assert kt.resolve_launches == 2 * ns
    assert kt.stage_matrices + kt.dependent_matrices == 2 * 2 * cfg.N
    assert kt.stage_matrices == 2 * 2 * sum(n for _, n in split)
    # look-ahead: a stage's independent visits may start beside the previous stage's
    assert 0 < kt.stage_union_ms <= kt.stage_ms * (1 + 1e-3) + 0.05
    P.ptca_set_launch_config(ctx.h, P.PIPELINE_GRAPH, 8, 0)
    ctx.sweep(1)
    assert P.ptca_kernel_times(ctx.h)[1] == 0               # one persistent launch: not per-stage
    P.ptca_set_kernel_timing(ctx.h, False)
    ctx.close()


@pytest.mark.parametrize("lat", [
    dict(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK),          # 4 stages
    dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6),                # ragged windows, 6 stages
    dict(Lx=24, Ly=1, L_c=4, schedule=P.SCHEDULE_BLOCK),            # chain: 2 stages
    dict(Lx=12, Ly=1, L_c=3, stride=3),                             # chain: 3 stages (copies wrap)
    dict(Lx=24, Ly=24, L_c=8, stride=8),                            # tiled: 64 stages of 9 sites
])
@pytest.mark.parametrize("margin", [1e-2, 50.0])
def test_overlapped_resolve_gives_the_one_stream_chain_bit_for_bit(lat, margin):
    """The overlapped pipeline against the one-stream per-stage pipeline:
    spins and every field of the per-visit record identical (F to the bit).
    margin 50 defers every decision, so every visit is re-solved while the
    next stage's independent visits run."""
    cfg = P.Config(**lat, T=0.1, mu=-6.5, seed=29, precision=P.MIXED, proposal=P.PROPOSAL_CONE)
    runs = []
    for mode in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP):
        ctx = P.Context(cfg)
        P.ptca_set_resolve_margin(ctx.h, margin)
        P.ptca_set_launch_config(ctx.h, mode, 8, 0)
        recs, stats = [], []
        for n in (1, 3, 2):
            st = ctx.sweep(n)
            stats.append((st.attempts, st.accepted, st.eigensolves))
            recs.append([x.cpu().numpy() for x in ctx.record()])
        runs.append((ctx.spins().cpu().numpy(), recs, stats))
        ctx.close()
    (S0, r0, t0), (S1, r1, t1) = runs
    assert t0 == t1
    assert np.array_equal(S0, S1)
    for a, b in zip(r0, r1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    # The same calls without statistics, back to back: each leaves its last
    # re-solve to the next, and the rotation runs on across the calls.
    ctx = P.Context(cfg)
    P.ptca_set_resolve_margin(ctx.h, margin)
    P.ptca_set_launch_config(ctx.h, P.PIPELINE_OVERLAP, 8, 0)
    for n in (1, 3, 2):
        P.ptca_sweep(ctx.h, n, stats=False)
    assert np.array_equal(ctx.spins().cpu().numpy(), S0)
    for x, y in zip([x.cpu().numpy() for x in ctx.record()], r0[-1]):
        assert np.array_equal(x, y)
    ctx.close()


@pytest.mark.parametrize("cfgkw", [
    dict(Lx=16, Ly=16, L_c=4, schedule=P.SCHEDULE_BLOCK, model=P.MODEL_HUBBARD_MF, U=8.0, mu=4.0, T=0.1),   # n = 32
    dict(Lx=128, Ly=1, L_c=8, stride=8, update_offset=4, model=P.MODEL_HOLSTEIN, lam=1.5, K=1.0, mu=0.0,
         T=0.1, m_step=0.4),                                                                                 # n = 16
])
def test_one_warp_ctas_compute_the_same_chain(cfgkw):
    # Matrices up to n = 32 also run one warp per matrix; with the guard the
    # chain (decisions, spins) is that of the wider CTAs in every pipeline.
    cfg = P.Config(**cfgkw, seed=21, precision=P.MIXED)
    runs = []
    for pl, nw in [(P.PIPELINE_STAGES, 8), (P.PIPELINE_STAGES, 1), (P.PIPELINE_OVERLAP, 1),
                   (P.PIPELINE_PERSISTENT, 1), (P.PIPELINE_GRAPH, 4)]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, pl, nw, 0)
        ctx.sweep(2)
        runs.append((ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    S0, (site, Fo, Fn, lnu, acc) = runs[0]
    for S, (site2, Fo2, Fn2, lnu2, acc2) in runs[1:]:
        assert np.array_equal(site, site2) and np.array_equal(acc, acc2)
        assert np.array_equal(S, S0)
        assert np.max(np.abs(Fo2 - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5
    # The one-warp per-stage and overlapped pipelines re-solve with the same
    # kernel: bit-identical.  (The persistent kernel re-solves inline at its
    # own CTA width, so its re-solved free energies agree only to rounding.)
    for a, b in zip(runs[1][1], runs[2][1]):
        assert np.array_equal(a, b)


def test_one_warp_width_is_limited_to_order_32():
    ctx = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.MIXED))   # n = 128
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 1, 0)
    ctx.close()
    ctx = P.Context(P.Config(Lx=8, Ly=8, L_c=4, precision=P.FP64))      # FP64
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 1, 0)
    ctx.close()


@pytest.mark.parametrize("kind,margin", [("n128", None), ("n128", 1e6), ("n288", None)])
def test_calls_that_leave_the_last_resolve_pending_compute_the_same_chain(kind, margin):
    # Overlapped pipeline: a call without statistics leaves its last stage's
    # re-solve for the next call.  Three such calls (the second on another
    # stream) must give the chain of one three-sweep call, and every entry
    # point that reads the configuration must see it complete.  margin 1e6:
    # every decision is re-solved, so the pending work is a whole stage.
    # n288: 12x12 clusters, the large-cluster kernel with its matrix-slot sets.
    if kind == "n128":
        cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=31,
                       precision=P.MIXED)
        width = 4
    else:
        cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=32,
                       precision=P.MIXED)
        width = 16

    def ctx_():
        c = P.Context(cfg)
        P.ptca_set_launch_config(c.h, P.PIPELINE_OVERLAP, width, 0)
        if margin is not None:
            P.ptca_set_resolve_margin(c.h, margin)
        return c

    a, b = ctx_(), ctx_()
    other = torch.cuda.Stream()
    P.ptca_sweep(a.h, 1, stats=False)
    P.ptca_sweep(a.h, 1, stats=False, stream=other)
    P.ptca_sweep(a.h, 1, stats=False)
    rec_a = [x.cpu().numpy() for x in a.record()]
    S_a = a.spins().cpu().numpy()
    st_b = b.sweep(3)
    rec_b = [x.cpu().numpy() for x in b.record()]
    assert np.array_equal(S_a, b.spins().cpu().numpy())
    for x, y in zip(rec_a, rec_b):
        assert np.array_equal(x, y)
    if margin is not None:
        assert st_b.resolved == 3 * cfg.N
    # one more pending call each, then statistics, observables and a flush
    P.ptca_sweep(a.h, 1, stats=False)
    P.ptca_sweep(b.h, 1, stats=False)
    P.ptca_flush(a.h)
    oa, ob = a.observables(), b.observables()
    assert (oa.S_pipi, oa.S_00, oa.F_site) == (ob.S_pipi, ob.S_00, ob.F_site)
    sa, sb = a.sweep(1), b.sweep(1)
    assert (sa.accepted, sa.resolved, sa.eigensolves) == (sb.accepted, sb.resolved, sb.eigensolves)
    assert np.array_equal(a.spins().cpu().numpy(), b.spins().cpu().numpy())
    a.close()
    b.close()

"""The shared reduction (launch configuration reduction =
PTCA_REDUCTION_SHARED: one 4-warp CTA per update site, FP32, orders up to
128).

H_new differs from H_old only in the update site's on-site block, so one
block Householder reduction in 2-column panels (Sec. II.c step b, blocked)
serves both matrices; each 2x2 block-tridiagonal form is then made
tridiagonal by a Givens bulge chase.  Checked against the oracle's solves of
every visit (free energies, ln u, decisions, spins) on full, clipped and
odd-sized windows, chains down to two-site windows, the Hubbard and
Holstein models and a cube; against the row-chunked pass (same chain); and on
the free-energy-difference scale at the headline size, where its error is
about twice the row-chunked pass's; the autotuner does not select it.

The large-cluster form (16-warp CTAs, the matrix in a global slot, chases in
double-float) against the oracle at n = 288, 512 and on clipped windows,
against the per-matrix large kernel (same chain), on dF against FP64 (far
below the per-matrix kernel's error), as the default of mixed large
contexts, and with its 1e-4 default re-solve margin."""
import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests import inputs
from tests.test_gpu_parity import _check_sweep_against_oracle
from tests.test_gpu_precision import MIXED_DF_BOUND, _level_scale

pytestmark = pytest.mark.gpu

SHARED_STAGES = (P.PIPELINE_STAGES, 4, 0, P.REDUCTION_SHARED)
SHARED_OVERLAP = (P.PIPELINE_OVERLAP, 4, 0, P.REDUCTION_SHARED)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


@pytest.mark.parametrize("lat", [
    dict(Lx=8, Ly=8, L_c=4),                                   # n = 32, corner-centred windows (tiled)
    dict(Lx=8, Ly=8, L_c=4, schedule=P.SCHEDULE_BLOCK),        # update site already first
    dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6),           # n = 18 .. 72, clipped windows
    dict(Lx=24, Ly=1, L_c=2, stride=2),                        # chain, n = 4: one panel
    dict(Lx=30, Ly=1, L_c=5, stride=5),                        # chain, n = 10
    dict(Lx=9, Ly=1, L_c=3, periodic=0, stride=3),             # open chain: windows of 2 and 3 sites
])
def test_shared_reduction_against_the_oracle_every_visit(lat):
    cfg = P.Config(**lat, t=1.0, J_H=8.0, mu=-6.5, T=0.05, seed=3, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, launch=SHARED_STAGES)


def test_shared_reduction_against_the_oracle_n128_overlap():
    # 24x24 torus, 8x8 clusters (n = 128: 63 panels), the paper's block
    # schedule, cone proposals: sampled visits plus those nearest the
    # Metropolis threshold (re-solved), through the overlapped pipeline.
    cfg = P.Config(Lx=24, Ly=24, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                   T=0.05, mu=-6.5, seed=9, precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=12, near=6, launch=SHARED_OVERLAP)


def test_shared_reduction_tiled_schedule_n128():
    # centred windows: the update site is moved to the front of the basis
    cfg = P.Config(Lx=24, Ly=24, L_c=8, schedule=P.SCHEDULE_TILED, stride=8, T=0.05, mu=-6.5, seed=5,
                   precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=16, near=4, launch=SHARED_STAGES)


def test_shared_reduction_hubbard_and_holstein():
    hub = P.Config(Lx=13, Ly=11, L_c=6, periodic=0, stride=6, t=1.0, U=8.0, mu=4.0, T=0.1, seed=3,
                   model=P.MODEL_HUBBARD_MF, m_step=0.5, precision=P.MIXED)
    _check_sweep_against_oracle(hub, sweeps=2, start=inputs.random_fields(61, hub.N, 2.0), launch=SHARED_STAGES)
    hol = P.Config(Lx=32, Ly=1, L_c=8, t=1.0, lam=1.5, K=1.0, mu=0.0, T=0.1, m_step=0.4, seed=2,
                   model=P.MODEL_HOLSTEIN, precision=P.MIXED)
    _check_sweep_against_oracle(hol, sweeps=2, launch=SHARED_STAGES)


def test_shared_reduction_cube():
    cfg = P.Config(Lx=8, Ly=8, Lz=8, L_c=4, schedule=P.SCHEDULE_BLOCK, T=0.1, mu=-6.5, seed=8,
                   precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=24, near=4, launch=SHARED_STAGES)


@pytest.mark.parametrize("lat", [dict(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK),
                                 dict(Lx=23, Ly=21, L_c=7, periodic=0, stride=7)])
def test_shared_and_row_chunked_reductions_compute_the_same_chain(lat):
    cfg = P.Config(**lat, proposal=P.PROPOSAL_CONE, T=0.05, mu=-6.5, seed=17, precision=P.MIXED)
    runs = []
    for launch in [(P.PIPELINE_STAGES, 4, 0, P.REDUCTION_ROWS), SHARED_STAGES, SHARED_OVERLAP]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, *launch)
        got = P.ptca_get_launch_config(ctx.h)
        assert (got.pipeline, got.warps_per_cta, got.ctas_per_sm, got.reduction) == launch
        stats = ctx.sweep(2)
        assert stats.eigensolves == 4 * cfg.N
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
    # the two shared pipelines run the same kernel on the same snapshots: bit for bit
    for x, y in zip(runs[1][1], runs[2][1]):
        assert np.array_equal(x, y)


# dF error bound of the shared reduction on the free-energy-difference scale.
# Its FP32 dF error is about twice the row-chunked pass's (whole headline
# stages against FP64: max |d dF| 1.6e-4 .. 2.2e-4 against 0.9e-4 .. 1.1e-4
# over four seeds).  Three times the row pass's bound.
SHARED_DF_BOUND = 3 * MIXED_DF_BOUND


def test_shared_dF_error_on_the_free_energy_difference_scale():
    # Stage 0 of the 100x100 headline, unguarded (margin 0): sampled visits'
    # dF against the oracle's, on the scale max(|dF|, sum_k |eps_k - mu| f_k / n).
    base = dict(Lx=100, Ly=100, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                T=0.05, mu=-6.5, seed=0)
    m = oracle.Model(Lx=100, Ly=100, Lc=8, JH=8.0, mu=-6.5, T=0.05, schedule=oracle.SCHEDULE_BLOCK,
                     proposal=oracle.PROPOSAL_CONE, cone_deg=30.0, seed=0)
    cfg = P.Config(**base, precision=P.MIXED)
    stage0 = P.ptca_schedule(cfg)[0]
    ctx = P.Context(cfg)
    P.ptca_set_launch_config(ctx.h, *SHARED_STAGES)
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
    assert worst <= SHARED_DF_BOUND, worst


def test_shared_reduction_configuration_is_validated():
    mixed = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.MIXED))
    for bad in [(P.PIPELINE_STAGES, 8, 0, P.REDUCTION_SHARED),       # 8-warp CTAs
                (P.PIPELINE_STAGES, 1, 0, P.REDUCTION_SHARED),       # one-warp CTAs
                (P.PIPELINE_PERSISTENT, 4, 0, P.REDUCTION_SHARED),   # persistent kernel
                (P.PIPELINE_GRAPH, 4, 0, P.REDUCTION_SHARED)]:
        with pytest.raises(P.PtcaError):
            P.ptca_set_launch_config(mixed.h, *bad)
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(mixed.h, P.PIPELINE_STAGES, 4, 0, 3)
    assert P.ptca_get_launch_config(mixed.h).reduction == P.REDUCTION_ROWS  # unchanged
    mixed.close()
    fp64 = P.Context(P.Config(Lx=16, Ly=16, L_c=8, precision=P.FP64))
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(fp64.h, *SHARED_STAGES)
    fp64.close()
    big = P.Context(P.Config(Lx=20, Ly=20, L_c=10, precision=P.MIXED))  # n = 200 > 128
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(big.h, *SHARED_STAGES)
    big.close()


def test_autotune_does_not_select_the_shared_reduction():
    # its larger dF error would narrow the re-solve guard's safety factor
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=23,
                   precision=P.MIXED)
    ctx = P.Context(cfg)
    best, table = P.ptca_autotune(ctx.h, 1)
    assert all(c["reduction"] != P.REDUCTION_SHARED for c in table["candidates"])
    assert best.reduction != P.REDUCTION_SHARED
    ctx.close()


# Large clusters (orders above the shared-memory kernels'): 16-warp CTAs with
# the matrix in a global slot.
LARGE_SHARED_STAGES = (P.PIPELINE_STAGES, 16, 0, P.REDUCTION_SHARED)
LARGE_SHARED_OVERLAP = (P.PIPELINE_OVERLAP, 16, 0, P.REDUCTION_SHARED)


@pytest.mark.parametrize("Lc,sample,near", [(12, 3, 2), (16, 1, 1)])
def test_large_shared_reduction_against_the_oracle(Lc, sample, near):
    # n = 288 and 512: sampled visits and the nearest to the threshold
    cfg = P.Config(Lx=2 * Lc, Ly=2 * Lc, L_c=Lc, schedule=P.SCHEDULE_BLOCK, J_H=8.0, mu=-6.5, T=0.1, seed=Lc,
                   precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=sample, near=near, launch=LARGE_SHARED_STAGES)


def test_large_shared_reduction_clipped_windows():
    # open lattice: windows of 9x9 .. 15x15 sites (n = 162 .. 450), ragged
    cfg = P.Config(Lx=33, Ly=31, L_c=15, periodic=0, stride=15, J_H=8.0, mu=-6.5, T=0.1, seed=4,
                   precision=P.MIXED)
    _check_sweep_against_oracle(cfg, sweeps=1, sample=2, launch=LARGE_SHARED_STAGES)


def test_large_shared_and_default_large_kernels_compute_the_same_chain():
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=5,
                   precision=P.MIXED)
    runs = []
    for launch in [(P.PIPELINE_STAGES, 16, 0, P.REDUCTION_ROWS), LARGE_SHARED_STAGES, LARGE_SHARED_OVERLAP]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, *launch)
        ctx.sweep(2)
        rec = [x.cpu().numpy() for x in ctx.record()]
        runs.append((ctx.spins().cpu().numpy(), rec))
        ctx.close()
    S_ref, (site, Fo, Fn, lnu, acc) = runs[0]
    for S, (site2, Fo2, Fn2, lnu2, acc2) in runs[1:]:
        assert np.array_equal(site, site2) and np.array_equal(acc, acc2)
        assert np.array_equal(S, S_ref)
        assert np.max(np.abs(Fo2 - Fo) / np.maximum(1.0, np.abs(Fo))) < 1e-5
        assert np.max(np.abs(Fn2 - Fn) / np.maximum(1.0, np.abs(Fn))) < 1e-5
    for x, y in zip(runs[1][1], runs[2][1]):
        assert np.array_equal(x, y)


def test_large_mixed_contexts_default_to_the_shared_reduction():
    # large clusters in PTCA_MIXED start on the shared reduction (faster than
    # the per-matrix kernel, and its dF error far smaller: its chases run in
    # double-float); FP64 contexts keep the per-matrix kernel; the autotuner
    # times both
    mixed = P.Context(P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED))
    got = P.ptca_get_launch_config(mixed.h)
    assert (got.pipeline, got.warps_per_cta, got.reduction) == (P.PIPELINE_STAGES, 16, P.REDUCTION_SHARED)
    best, table = P.ptca_autotune(mixed.h, 1)
    shared = [c for c in table["candidates"] if c["reduction"] == P.REDUCTION_SHARED]
    assert {c["pipeline"] for c in shared} == {"stages", "overlap"}
    assert all(c["ms_per_sweep"] is not None for c in shared)
    mixed.close()
    fp64 = P.Context(P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, precision=P.FP64))
    assert P.ptca_get_launch_config(fp64.h).reduction == P.REDUCTION_ROWS
    with pytest.raises(P.PtcaError):
        P.ptca_set_launch_config(fp64.h, *LARGE_SHARED_STAGES)
    fp64.close()


def test_large_shared_dF_error_is_far_below_the_per_matrix_kernels():
    # Stage 0 of a 48x48 torus with 12x12 clusters (n = 288), unguarded:
    # dF against the FP64 path on the same start, every visit of the stage.
    # The shared reduction's FP32 rounding is common to both matrices and its
    # chases run in double-float (measured max 4.6e-7 against 2.0e-4 for the
    # per-matrix kernel).
    base = dict(Lx=48, Ly=48, L_c=12, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, cone_deg=30.0,
                T=0.05, mu=-6.5, seed=1)
    n0 = len(P.ptca_schedule(P.Config(**base, precision=P.FP64))[0])
    ref = P.Context(P.Config(**base, precision=P.FP64))
    ref.sweep(1)
    _, Fo64, Fn64, _, _ = (x.cpu().numpy()[:n0] for x in ref.record())
    ref.close()
    err = {}
    for red in (P.REDUCTION_ROWS, P.REDUCTION_SHARED):
        ctx = P.Context(P.Config(**base, precision=P.MIXED))
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 16, 0, red)
        P.ptca_set_resolve_margin(ctx.h, 0.0)
        ctx.sweep(1)
        _, Fo, Fn, _, _ = (x.cpu().numpy()[:n0] for x in ctx.record())
        ctx.close()
        err[red] = np.max(np.abs((Fn - Fo) - (Fn64 - Fo64)))
    assert err[P.REDUCTION_SHARED] < 5e-6
    assert err[P.REDUCTION_SHARED] < 0.05 * err[P.REDUCTION_ROWS]


def test_large_shared_default_margin_follows_the_launch_configuration():
    # n = 288: the shared reduction's default re-solve margin is 1e-4 (its dF
    # error is about 5e-7); a margin the caller sets is kept across launch
    # configurations.  Runs compare bit for bit against explicit margins.
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, proposal=P.PROPOSAL_CONE, T=0.05, seed=6,
                   precision=P.MIXED)

    def run(setup):
        ctx = P.Context(cfg)
        setup(ctx)
        st = ctx.sweep(2)
        rec = [x.cpu().numpy() for x in ctx.record()]
        ctx.close()
        return st.resolved, rec

    r_default, rec_default = run(lambda c: None)
    r_1e4, rec_1e4 = run(lambda c: P.ptca_set_resolve_margin(c.h, 1e-4))
    assert r_default == r_1e4
    for x, y in zip(rec_default, rec_1e4):
        assert np.array_equal(x, y)

    def switch(c):  # through the per-matrix kernel and back: the default follows
        P.ptca_set_launch_config(c.h, P.PIPELINE_STAGES, 16, 0, P.REDUCTION_ROWS)
        P.ptca_set_launch_config(c.h, *LARGE_SHARED_STAGES)
    r_switch, rec_switch = run(switch)
    assert r_switch == r_default
    for x, y in zip(rec_default, rec_switch):
        assert np.array_equal(x, y)

    def user_margin(c):  # set by the caller: kept
        P.ptca_set_resolve_margin(c.h, 1e-2)
        P.ptca_set_launch_config(c.h, *LARGE_SHARED_STAGES)
    r_user, _ = run(user_margin)
    assert r_user >= r_default


def test_persistent_pipelines_return_large_contexts_to_the_per_matrix_reduction():
    # The persistent kernels reduce one matrix at a time: selecting one with
    # ptca_set_pipeline resets the reduction, and the sweep matches the
    # per-stage per-matrix sweep bit for bit (every decision re-solved, as in
    # the large-cluster pipeline tests).
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, T=0.1, seed=7, precision=P.MIXED,
                   proposal=P.PROPOSAL_CONE)
    ref = P.Context(cfg)
    P.ptca_set_launch_config(ref.h, P.PIPELINE_STAGES, 16, 0, P.REDUCTION_ROWS)
    P.ptca_set_resolve_margin(ref.h, 1e6)
    ref.sweep(1)
    rec_ref = [x.cpu().numpy() for x in ref.record()]
    S_ref = ref.spins().cpu().numpy()
    ref.close()
    ctx = P.Context(cfg)
    assert P.ptca_get_launch_config(ctx.h).reduction == P.REDUCTION_SHARED
    P.ptca_set_resolve_margin(ctx.h, 1e6)
    P.ptca_set_pipeline(ctx.h, P.PIPELINE_PERSISTENT)
    got = P.ptca_get_launch_config(ctx.h)
    assert (got.pipeline, got.reduction) == (P.PIPELINE_PERSISTENT, P.REDUCTION_ROWS)
    ctx.sweep(1)
    assert np.array_equal(ctx.spins().cpu().numpy(), S_ref)
    for x, y in zip(rec_ref, (r.cpu().numpy() for r in ctx.record())):
        assert np.array_equal(x, y)
    ctx.close()

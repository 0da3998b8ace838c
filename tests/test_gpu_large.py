"""Large traveling clusters (the paper's N_c = 12^2 and 16^2, Sec. VII.a):
matrix orders above the shared-memory kernels' (200 ... 512) run on the
global-memory Householder path with 16-warp CTAs, or on thread-block
clusters.  Sweeps against the oracle visit by visit in FP64 and mixed
precision; bit identity of the per-stage, overlapped and persistent
pipelines; the precision checker and the batch eigenvalue call at these
orders."""
import numpy as np
import pytest
import torch

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
    assert P.ptca_get_launch_config(ctx.h).pipeline == P.PIPELINE_STAGES  # the large-cluster default
    for pl in (P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH):
        with pytest.raises(P.PtcaError) as e:
            P.ptca_set_launch_config(ctx.h, pl, 8, 0)  # the cluster kernel has no persistent form
        assert e.value.status in (1, 6)
    with pytest.raises(P.PtcaError) as e:
        P.ptca_set_launch_config(ctx.h, P.PIPELINE_STAGES, 4, 0)
    assert e.value.status == 6
    assert P.ptca_get_launch_config(ctx.h).warps_per_cta == 16
    best, table = P.ptca_autotune(ctx.h, 1)
    timed = {(c["pipeline"], c["warps_per_cta"]) for c in table["candidates"] if c["ms_per_sweep"] is not None}
    assert {("stages", 16), ("overlap", 16), ("persistent", 16), ("graph", 16)} <= timed
    ctx.close()


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
def test_large_cluster_persistent_pipelines_are_bit_identical(prec):
    # 24x24 torus, 12x12 clusters (n = 288): the persistent launch (and its
    # CUDA graph) against per-stage launches, two one-sweep calls; in
    # PTCA_MIXED with every decision re-solved inline by the persistent kernel.
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, T=0.1, seed=4, precision=prec,
                   proposal=P.PROPOSAL_CONE)
    runs = []
    for pl in (P.PIPELINE_STAGES, P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH):
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, pl, 16, 0)
        if prec == P.MIXED:
            P.ptca_set_resolve_margin(ctx.h, 1e6)
        recs = []
        for _ in range(2):
            st = ctx.sweep(1)
            assert st.attempts == cfg.N
            if prec == P.MIXED:
                assert st.resolved == cfg.N
            recs.append([x.cpu().numpy() for x in ctx.record()])
        runs.append((ctx.spins().cpu().numpy(), recs))
        ctx.close()
    for S, recs in runs[1:]:
        assert np.array_equal(runs[0][0], S)
        for a, b in zip(runs[0][1], recs):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_large_cluster_precision_checker():
    # The checker on 12x12 clusters (n = 288): FP32 against FP64 spectra of
    # every visit of a sweep, in the context's global slots.  The chain is
    # unchanged by it.
    cfg = P.Config(Lx=24, Ly=24, L_c=12, schedule=P.SCHEDULE_BLOCK, T=0.05, seed=6, precision=P.MIXED,
                   proposal=P.PROPOSAL_CONE)
    ctx = P.Context(cfg)
    P.ptca_set_checker(ctx.h, True)
    ctx.sweep(1)
    rows = P.ptca_checker_read(ctx.h, 4)
    S = ctx.spins().cpu().numpy()
    ctx.close()
    assert rows.shape == (4, 5) and np.all(np.isfinite(rows))
    assert np.all(rows[:, 0] > 0)                 # the FP32 reduction is not exact
    assert rows[:, 2].max() < 1e-5                # eigenvalue error / (J_H + 4|t|)
    assert rows[:, 4].max() < 2e-3                # dF error on the dF scale at n = 288
    ref = P.Context(cfg)
    ref.sweep(1)
    assert np.array_equal(ref.spins().cpu().numpy(), S)
    ref.close()


@pytest.mark.parametrize("prec,tol", [(P.FP64, 1e-11), (P.MIXED, 2e-5)])
def test_large_cluster_batch_eigenvalues(prec, tol):
    # Clusters of a 12x12 window (n = 288) and clipped windows near the corner
    # (n = 72, 198) of an open lattice, built by the library; their eigenvalues against
    # LAPACK on the host (numpy.linalg.eigvalsh of the same matrices read back).
    cfg = P.Config(Lx=24, Ly=24, L_c=12, periodic=0, stride=12, T=0.1, seed=2, precision=prec)
    ctx = P.Context(cfg)
    ctx.set_spins(inputs.random_unit_spins(5, cfg.N))
    H, offs, n = ctx.build_clusters([12 * 24 + 12, 0, 5 * 24 + 3])
    eig, _ = ctx.cluster_eigvals(H, offs, n)
    n_host = n.cpu().numpy()
    assert n_host.max() == 288 and n_host.min() < 288
    Hh = H.cpu().numpy().astype(np.complex128)
    o = offs.cpu().numpy()
    e = eig.cpu().numpy()
    for i, k in enumerate(n_host):
        k = int(k)
        A = np.zeros((k, k), dtype=np.complex128)
        r, c = np.tril_indices(k)
        A[r, c] = Hh[o[i]:o[i] + k * (k + 1) // 2]
        A = A + np.tril(A, -1).conj().T
        want = np.linalg.eigvalsh(A)
        assert np.max(np.abs(e[i, :k] - want)) <= tol * max(1.0, np.abs(want).max()), i
    ctx.close()

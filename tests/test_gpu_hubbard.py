"""GPU parity of the Hubbard mean-field model (Eq. 1 with <n_i> = 1) against
the oracle: the batch builder's matrices, whole sweeps visit by visit (F_old,
F_new with the window's classical energy, ln u, decisions, the replayed
configuration), the decisions of a sequential oracle sweep in FP64, and the
overlapped pipeline's bit identity.  Fields start with lengths spread over
[0, 2] so the variable-magnitude terms are exercised."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests import inputs
from tests.test_gpu_parity import _check_sweep_against_oracle, _oracle_model, _unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _cfg(**kw):
    base = dict(Lx=8, Ly=8, L_c=4, t=1.0, U=8.0, mu=4.0, T=0.1, seed=3, model=P.MODEL_HUBBARD_MF, m_step=0.5)
    base.update(kw)
    return P.Config(**base)


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
def test_build_clusters_matches_oracle(prec):
    cfg = _cfg(Lx=12, Ly=11, L_c=6, periodic=0, stride=6, precision=prec)
    ctx = P.Context(cfg)
    S = inputs.random_fields(51, cfg.N, 2.0)
    ctx.set_spins(S)
    sites = np.arange(cfg.N, dtype=np.int32)[::7]
    new = inputs.random_fields(52, sites.size, 2.0)
    m = _oracle_model(cfg)
    for use_new in (False, True):
        H, offs, n = ctx.build_clusters(sites, new if use_new else None)
        H, offs, n = H.cpu().numpy(), offs.cpu().numpy(), n.cpu().numpy()
        for i, s in enumerate(sites):
            ref, _ = oracle.cluster_hamiltonian(m, S, int(s), new[i] if use_new else None)
            mine = _unpack(H[offs[i]: offs[i] + n[i] * (n[i] + 1) // 2].astype(np.complex128), n[i])
            tol = 1e-14 * 16.0 if prec == P.FP64 else 1e-6 * 16.0
            assert np.max(np.abs(mine - ref)) <= tol
    ctx.close()


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
@pytest.mark.parametrize("lat", [dict(Lx=8, Ly=8, L_c=4),
                                 dict(Lx=16, Ly=16, L_c=8, schedule=P.SCHEDULE_BLOCK),
                                 dict(Lx=13, Ly=11, L_c=6, periodic=0, stride=6)])
def test_sweeps_match_oracle_visit_by_visit(prec, lat):
    cfg = _cfg(**lat, precision=prec)
    start = inputs.random_fields(60 + cfg.Lx, cfg.N, 2.0)
    sample = None if cfg.N <= 64 else 40
    _check_sweep_against_oracle(cfg, sweeps=2, sample=sample, start=start)


def test_fp64_sweeps_equal_the_sequential_oracle_sweep():
    cfg = _cfg(precision=P.FP64, T=0.2, m_step=0.8)
    ctx = P.Context(cfg)
    m = _oracle_model(cfg)
    S = inputs.random_fields(70, cfg.N, 1.5)
    ctx.set_spins(S)
    for sw in range(4):
        ctx.sweep(1)
        site, Fo, Fn, lnu, acc = (x.cpu().numpy() for x in ctx.record())
        S_ref, rec = oracle.sweep(m, S, sw)
        assert np.array_equal(site, rec.site)
        assert np.max(np.abs(Fo - rec.F_old) / np.maximum(1.0, np.abs(rec.F_old))) < 1e-9
        assert np.max(np.abs(Fn - rec.F_new) / np.maximum(1.0, np.abs(rec.F_new))) < 1e-9
        margin = np.abs(rec.lnu + (rec.F_new - rec.F_old) / cfg.T)
        sure = margin > 1e-6
        assert np.array_equal(acc[sure].astype(bool), rec.accepted[sure].astype(bool))
        S = ctx.spins().cpu().numpy()
        if np.all(sure):
            assert np.max(np.abs(S - S_ref)) < 1e-12
    ctx.close()


def test_overlap_pipeline_is_bit_identical_and_fields_change_length():
    cfg = _cfg(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED, T=0.2)
    start = inputs.random_fields(80, cfg.N, 2.0)
    runs = []
    for pl in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP, P.PIPELINE_GRAPH):
        ctx = P.Context(cfg)
        ctx.set_spins(start)
        P.ptca_set_launch_config(ctx.h, pl, 8, 0)
        ctx.sweep(2)
        runs.append((ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    for S, rec in runs[1:]:
        assert np.array_equal(S, runs[0][0])
        for a, b in zip(rec, runs[0][1]):
            assert np.array_equal(a, b)
    r0 = np.linalg.norm(start, axis=1)
    r1 = np.linalg.norm(runs[0][0], axis=1)
    moved = np.abs(r1 - r0) > 1e-9
    assert moved.mean() > 0.3                     # lengths are sampled, not fixed
    assert np.all(np.abs(r1 - r0) <= 2 * 0.5 + 1e-12)   # at most two steps of m_step


def test_surrogate_is_refused_for_the_hubbard_model():
    ctx = P.Context(_cfg(precision=P.MIXED))
    with pytest.raises(P.PtcaError) as e:
        P.ptca_surrogate_init(ctx.h, 1)
    assert e.value.status == 6
    ctx.close()

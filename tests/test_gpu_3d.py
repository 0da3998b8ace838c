"""GPU parity on cubic lattices (Lz > 1): the paper's 3-D workloads with
4^3 traveling clusters (n = 128) and eight blocks (Sec. III.a, IV).  The
batch builder's matrices, whole sweeps visit by visit against the oracle for
both models and precisions, pipeline bit identity, and S(q) at (pi,pi,pi)."""
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


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
@pytest.mark.parametrize("lat", [dict(Lx=8, Ly=8, Lz=8, L_c=4), dict(Lx=7, Ly=6, Lz=5, L_c=3, periodic=0, stride=3)])
def test_build_clusters_matches_oracle(prec, lat):
    cfg = P.Config(**lat, precision=prec)
    ctx = P.Context(cfg)
    S = inputs.random_unit_spins(90, cfg.N)
    ctx.set_spins(S)
    sites = np.arange(cfg.N, dtype=np.int32)[:: max(1, cfg.N // 19)]
    new = inputs.random_unit_spins(91, sites.size)
    m = _oracle_model(cfg)
    for use_new in (False, True):
        H, offs, n = ctx.build_clusters(sites, new if use_new else None)
        H, offs, n = H.cpu().numpy(), offs.cpu().numpy(), n.cpu().numpy()
        for i, s in enumerate(sites):
            ref, _ = oracle.cluster_hamiltonian(m, S, int(s), new[i] if use_new else None)
            assert n[i] == ref.shape[0]
            mine = _unpack(H[offs[i]: offs[i] + n[i] * (n[i] + 1) // 2].astype(np.complex128), n[i])
            tol = 0.0 if prec == P.FP64 else 1e-6 * 8.0
            assert np.max(np.abs(mine - ref)) <= tol
    ctx.close()


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
@pytest.mark.parametrize("lat", [dict(Lx=8, Ly=8, Lz=8, L_c=4, schedule=P.SCHEDULE_BLOCK),
                                 dict(Lx=6, Ly=6, Lz=6, L_c=3, stride=3)])
def test_double_exchange_sweeps_match_oracle(prec, lat):
    cfg = P.Config(**lat, J_H=8.0, mu=-6.5, T=0.1, seed=4, precision=prec, proposal=P.PROPOSAL_CONE)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=40)


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
def test_hubbard_sweeps_match_oracle(prec):
    # The paper's 3-D benchmark model (Eq. 1): 8^3 torus, 4^3 clusters, U = 8.
    cfg = P.Config(Lx=8, Ly=8, Lz=8, L_c=4, schedule=P.SCHEDULE_BLOCK, model=P.MODEL_HUBBARD_MF, U=8.0, mu=4.0,
                   T=0.15, m_step=0.5, seed=6, precision=prec)
    start = inputs.random_fields(92, cfg.N, 2.0)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=40, start=start)


def test_pipelines_bit_identical_on_a_cube():
    cfg = P.Config(Lx=8, Ly=8, Lz=8, L_c=4, schedule=P.SCHEDULE_BLOCK, T=0.1, seed=8, precision=P.MIXED,
                   proposal=P.PROPOSAL_CONE)
    runs = []
    for pl, nw in [(P.PIPELINE_STAGES, 8), (P.PIPELINE_OVERLAP, 8), (P.PIPELINE_GRAPH, 8), (P.PIPELINE_OVERLAP, 4)]:
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, pl, nw, 0)
        ctx.sweep(2)
        runs.append((nw, ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    for nw, S, rec in runs[1:]:
        assert np.array_equal(S, runs[0][1])
        if nw == 8:
            for a, b in zip(rec, runs[0][2]):
                assert np.array_equal(a, b)


def test_structure_factor_at_pi_pi_pi():
    L = 8
    cfg = P.Config(Lx=L, Ly=L, Lz=L, L_c=4, schedule=P.SCHEDULE_BLOCK)
    ctx = P.Context(cfg)
    idx = np.arange(cfg.N)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    neel = np.where((x + y + z) % 2 == 0, 1.0, -1.0)[:, None] * np.array([0.6, 0.0, 0.8])
    ctx.set_spins(neel)
    o = P.ptca_observables(ctx.h)
    assert abs(o.S_pipi - 1.0) < 1e-12 and abs(o.S_00) < 1e-12
    R = inputs.random_unit_spins(93, cfg.N)
    ctx.set_spins(R)
    o = P.ptca_observables(ctx.h)
    ref = oracle.structure_factor(L, L, R, math.pi, math.pi, Lz=L, qz=math.pi)
    assert abs(o.S_pipi - ref) < 1e-12
    ctx.close()


def test_surrogate_is_refused_on_a_cube():
    ctx = P.Context(P.Config(Lx=8, Ly=8, Lz=8, L_c=4, precision=P.MIXED))
    with pytest.raises(P.PtcaError) as e:
        P.ptca_surrogate_init(ctx.h, 1)
    assert e.value.status == 6
    ctx.close()

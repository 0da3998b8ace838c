"""GPU parity of the adiabatic Holstein model (Sec. VII.b) against the
oracle: the initial distortions, sweeps visit by visit on the paper's chain
(N = 32, N_c = 8) with the 'corner' and 'central' update sites in FP64 and
mixed precision, a two-dimensional case, pipeline bit identity, and the
charge structure factor N(pi)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from paper_1502_07028_gb300 import _build
from tests import inputs
from tests.test_gpu_parity import _check_sweep_against_oracle, _oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _cfg(**kw):
    base = dict(Lx=32, Ly=1, L_c=8, t=1.0, lam=1.5, K=1.0, mu=0.0, T=0.1, m_step=0.4, seed=2,
                model=P.MODEL_HOLSTEIN)
    base.update(kw)
    return P.Config(**base)


def test_initial_distortions_equal_the_oracle():
    cfg = _cfg(Lx=512)
    ctx = P.Context(cfg)
    assert np.array_equal(ctx.spins().cpu().numpy(), oracle.init_spins(_oracle_model(cfg)))
    ctx.close()


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
@pytest.mark.parametrize("scheme", [dict(schedule=P.SCHEDULE_BLOCK, update_offset=0),       # corner
                                    dict(schedule=P.SCHEDULE_TILED, stride=8, update_offset=4)])  # central
def test_chain_sweeps_match_oracle(prec, scheme):
    cfg = _cfg(**scheme, precision=prec)
    _check_sweep_against_oracle(cfg, sweeps=3)


@pytest.mark.parametrize("prec", [P.FP64, P.MIXED])
def test_square_lattice_sweeps_match_oracle(prec):
    cfg = _cfg(Lx=12, Ly=12, L_c=4, schedule=P.SCHEDULE_BLOCK, lam=2.0, K=1.5, T=0.2, precision=prec)
    _check_sweep_against_oracle(cfg, sweeps=2, sample=40)


def test_pipelines_bit_identical():
    cfg = _cfg(Lx=256, schedule=P.SCHEDULE_BLOCK, precision=P.MIXED)
    runs = []
    for pl in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP, P.PIPELINE_GRAPH):
        ctx = P.Context(cfg)
        P.ptca_set_launch_config(ctx.h, pl, 8, 0)
        ctx.sweep(3)
        runs.append((ctx.spins().cpu().numpy(), [x.cpu().numpy() for x in ctx.record()]))
        ctx.close()
    for S, rec in runs[1:]:
        assert np.array_equal(S, runs[0][0])
        for a, b in zip(rec, runs[0][1]):
            assert np.array_equal(a, b)
    assert np.all(runs[0][0][:, 1:] == 0.0)   # only the distortion component moves


def test_charge_structure_factor():
    cfg = _cfg(Lx=64)
    ctx = P.Context(cfg)
    x = np.zeros((cfg.N, 3))
    x[:, 0] = np.where(np.arange(cfg.N) % 2 == 0, 1.3, -0.7)
    ctx.set_spins(x)
    o = P.ptca_observables(ctx.h)
    ref = oracle.structure_factor(cfg.N, 1, x, math.pi, 0.0)
    assert abs(o.S_pipi - ref) < 1e-12 and abs(ref - 1.0) < 1e-12
    ctx.close()

"""Stage pipeline (persistent launch, device-wide barrier, CUDA graph) and
ragged window sizes.

The three launch modes must give bit-identical sweeps: they run the same
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
    for mode in (P.PIPELINE_STAGES, P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH):
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
    for mode in (P.PIPELINE_PERSISTENT, P.PIPELINE_GRAPH):
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

"""Surrogate network and delayed acceptance on the GPU.

* forward values and gradients of the library's BF16 tensor-core kernels
  against the FP64 reference network (oracle/surrogate.py), which rounds the
  same operands to bfloat16;
* collected training inputs against patches recomputed from the stage-start
  spins;
* training lowers the loss and predicts held-out dF;
* delayed acceptance samples the same distribution as plain Metropolis, with
  a trained and with an untrained network (observables within 2 sigma);
* screened sweeps are the same chain in the one-stream and the overlapped
  per-stage pipelines, whatever the CTA width;
* the trained network saves exact cluster solves.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1502_07028_gb300 as P
from oracle import surrogate as SR
from paper_1502_07028_gb300 import _build
from tests import inputs
from tests.test_gpu_parity import _replay

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    assert torch.cuda.is_available()
    P.lib()


def _rand_samples(seed, n):
    spins = inputs.random_unit_spins(seed, n * 50).reshape(n, 50, 3)
    feat = np.concatenate([spins[:, :49, :].reshape(n, 147), spins[:, 49, :]], axis=1).astype(np.float32)
    center = inputs.rng(seed + 1).integers(0, 49, size=n).astype(np.int32)
    dF = inputs.rng(seed + 2).normal(scale=0.5, size=n).astype(np.float32)
    return feat, center, dF


def _params(ctx):
    theta = torch.empty(P.ptca_surrogate_param_count(), dtype=torch.float32, device="cuda")
    scale = P.ptca_surrogate_get_params(ctx.h, theta)
    return theta.cpu().numpy().astype(np.float64), scale


@pytest.mark.parametrize("n", [96, 700])
def test_forward_matches_bf16_reference(n):
    # 2n network rows: one or several 128-row tiles of the tensor-core
    # forward products, the last one ragged; K = 160 (zero-padded to three
    # 64-wide blocks) and 256; output widths 256 and 8.
    ctx = P.Context(P.Config(Lx=16, Ly=16, L_c=8))
    P.ptca_surrogate_init(ctx.h, 11)
    feat, center, _ = _rand_samples(3, n)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    P.ptca_surrogate_predict(ctx.h, torch.from_numpy(feat).cuda(), torch.from_numpy(center).cuda(), n, out)
    got = out.cpu().numpy().astype(np.float64)
    theta, scale = _params(ctx)
    ref = SR.surrogate_dF(theta, feat.astype(np.float64), center, scale)
    err = np.abs(got - ref)
    assert np.max(err) <= 2e-2 * np.max(np.abs(ref)), (np.max(err), np.max(np.abs(ref)))
    assert np.mean(err) <= 2e-3 * np.mean(np.abs(ref))
    ctx.close()


def test_gradients_match_fp64_reference():
    ctx = P.Context(P.Config(Lx=16, Ly=16, L_c=8))
    P.ptca_surrogate_init(ctx.h, 12)
    feat, center, dF = _rand_samples(5, 64)
    g = torch.empty(P.ptca_surrogate_param_count(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    P.ptca_surrogate_grad(ctx.h, torch.from_numpy(feat).cuda(), torch.from_numpy(center).cuda(),
                          torch.from_numpy(dF).cuda(), 64, g, loss)
    theta, scale = _params(ctx)
    ref_loss, ref_g = SR.loss_and_grad(theta, feat.astype(np.float64), center, dF.astype(np.float64), scale)
    assert abs(loss.item() - ref_loss) <= 1e-3 * ref_loss
    gg = g.cpu().numpy().astype(np.float64)
    for name, shp in SR.SHAPES:
        off = sum(int(np.prod(s)) for n, s in SR.SHAPES[: [n for n, _ in SR.SHAPES].index(name)])
        sl = slice(off, off + int(np.prod(shp)))
        num = np.linalg.norm(gg[sl] - ref_g[sl])
        den = np.linalg.norm(ref_g[sl]) + 1e-30
        if den > 1e-12:
            assert num / den <= 2e-2, (name, num / den)
    ctx.close()


@pytest.mark.parametrize("schedule", ["tiled", "block"])
def test_collected_inputs_are_window_patches(schedule):
    # 16x16 torus, 8x8 periodic clusters.  The patch is centred on the update
    # site and wraps inside the window: for the tiled schedule (update site at
    # window offset 4) that is the lattice neighbourhood; for the block
    # schedule (update site at the window's corner) the cluster's own wrap.
    kw = dict(stride=8) if schedule == "tiled" else dict(schedule=P.SCHEDULE_BLOCK)
    cfg = P.Config(Lx=16, Ly=16, L_c=8, T=0.1, seed=2, precision=P.FP64, **kw)
    ctx = P.Context(cfg)
    N = cfg.N
    S0 = ctx.spins().cpu().numpy()
    feat = torch.empty((N, 150), dtype=torch.float32, device="cuda")
    center = torch.empty(N, dtype=torch.int32, device="cuda")
    dF = torch.empty(N, dtype=torch.float32, device="cuda")
    P.ptca_surrogate_collect(ctx.h, 1, feat, center, dF)
    site, Fo, Fn, lnu, acc = (x.cpu().numpy() for x in ctx.record())
    stages = P.ptca_schedule(cfg)
    starts, _ = _replay(cfg, S0, stages, site, acc, 0)
    stage_of = np.zeros(N, dtype=np.int64)
    for k, st in enumerate(stages):
        stage_of[st] = k
    feat, center, dF = feat.cpu().numpy(), center.cpu().numpy(), dF.cpu().numpy()
    o = 4 if schedule == "tiled" else 0
    m = oracle.Model(Lx=16, Ly=16, Lc=8, stride=8 if schedule == "tiled" else 0, seed=2, T=0.1,
                     schedule=oracle.SCHEDULE_TILED if schedule == "tiled" else oracle.SCHEDULE_BLOCK)
    for k in range(0, N, 17):
        s = int(site[k])
        cx, cy = s % 16, s // 16
        Sst = starts[stage_of[s]]

        def lat(c, d):   # lattice coordinate of patch offset d (window start c - o)
            return (c - o + (o - 3 + d) % 8) % 16

        want = np.array([Sst[lat(cy, b) * 16 + lat(cx, a)] for b in range(7) for a in range(7)])
        assert center[k] == 24
        assert np.array_equal(feat[k, :147], want.astype(np.float32).ravel())
        assert np.array_equal(feat[k, 147:], oracle.propose(m, 0, s, Sst[s]).astype(np.float32))
        assert dF[k] == np.float32(Fn[k] - Fo[k])
    ctx.close()


@pytest.fixture(scope="module")
def trained():
    """A network trained on 32x32 exact sweeps (sphere proposals, T = 0.05),
    85% of the visits for training and a random 15% held out."""
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, T=0.05, mu=-6.5, seed=4, precision=P.MIXED)
    ctx = P.Context(cfg)
    sweeps = 48
    N = cfg.N
    feat = torch.empty((sweeps * N, 150), dtype=torch.float32, device="cuda")
    center = torch.empty(sweeps * N, dtype=torch.int32, device="cuda")
    dF = torch.empty(sweeps * N, dtype=torch.float32, device="cuda")
    P.ptca_surrogate_collect(ctx.h, sweeps, feat, center, dF)
    perm = torch.from_numpy(inputs.rng(8).permutation(sweeps * N)).cuda()
    ntr = int(0.85 * sweeps * N)
    tr, ho = perm[:ntr], perm[ntr:]
    ftr, ctr, dtr = feat[tr].contiguous(), center[tr].contiguous(), dF[tr].contiguous()
    P.ptca_surrogate_init(ctx.h, 1)
    steps = 1500
    loss = torch.empty(steps, dtype=torch.float32, device="cuda")
    P.ptca_surrogate_train(ctx.h, ftr, ctr, dtr, ntr, steps, 512, 1e-3, 1e-4, 7, loss)
    theta = torch.empty(P.ptca_surrogate_param_count(), dtype=torch.float32, device="cuda")
    scale = P.ptca_surrogate_get_params(ctx.h, theta)
    pred = torch.empty(ho.numel(), dtype=torch.float32, device="cuda")
    P.ptca_surrogate_predict(ctx.h, feat[ho].contiguous(), center[ho].contiguous(), ho.numel(), pred)
    out = dict(cfg=cfg, theta=theta, scale=scale, loss=loss.cpu().numpy(), pred=pred.cpu().numpy(),
               truth=dF[ho].cpu().numpy())
    ctx.close()
    return out


def test_training_lowers_loss_and_predicts_held_out(trained):
    loss = trained["loss"]
    assert np.mean(loss[-100:]) < 0.35 * np.mean(loss[:20]), (np.mean(loss[:20]), np.mean(loss[-100:]))
    r = np.corrcoef(trained["pred"], trained["truth"])[0, 1]
    assert r > 0.8, r


def _chain(cfg, sweeps, theta=None, scale=None, seed_net=None):
    ctx = P.Context(cfg)
    if theta is not None:
        P.ptca_surrogate_set_params(ctx.h, theta, scale)
        P.ptca_surrogate_enable(ctx.h, True)
    elif seed_net is not None:
        P.ptca_surrogate_init(ctx.h, seed_net)
        P.ptca_surrogate_enable(ctx.h, True)
    obs, solves, screened = [], 0, 0
    for _ in range(sweeps):
        st = ctx.sweep(1)
        solves += st.eigensolves
        screened += st.screened
        o = ctx.observables()
        obs.append((o.S_pipi, o.S_00))
    ctx.close()
    return np.array(obs), solves, screened


def _batch_z(a, b, nb=40):
    def mean_err(x):
        xb = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
        return xb.mean(), xb.std(ddof=1) / math.sqrt(nb)
    ma, ea = mean_err(a)
    mb, eb = mean_err(b)
    return (ma - mb) / math.sqrt(ea * ea + eb * eb + 1e-30)


@pytest.mark.parametrize("kind", ["untrained", "trained"])
def test_delayed_acceptance_samples_the_same_distribution(kind, trained):
    # 8x8 torus, 4x4 clusters, sphere proposals; chains of 2400 sweeps
    # (first 400 discarded) with plain Metropolis and with the screen.
    cfg = P.Config(Lx=8, Ly=8, L_c=4, T=0.3, mu=-6.5, seed=21, precision=P.MIXED)
    ref, solves_ref, _ = _chain(cfg, 2400)
    if kind == "untrained":
        da, solves_da, scr = _chain(P.Config(**{**cfg.__dict__, "seed": 22}), 2400, seed_net=99)
    else:
        da, solves_da, scr = _chain(P.Config(**{**cfg.__dict__, "seed": 22}), 2400, theta=trained["theta"],
                                    scale=trained["scale"])
    for q in range(2):
        z = _batch_z(ref[400:, q], da[400:, q])
        assert abs(z) < 2.0, (kind, q, z, ref[400:, q].mean(), da[400:, q].mean())
    assert scr > 0


def test_trained_network_saves_exact_solves(trained):
    # Same lattice, temperature and proposals as the training data.
    cfg = trained["cfg"]
    base, solves_base, _ = _chain(cfg, 6)
    da, solves_da, screened = _chain(cfg, 6, theta=trained["theta"], scale=trained["scale"])
    assert screened > 0
    assert solves_da < 0.8 * solves_base, (solves_da, solves_base)


@pytest.mark.parametrize("proposal", [P.PROPOSAL_SPHERE, P.PROPOSAL_CONE])
def test_screened_sweeps_are_one_chain_in_every_per_stage_pipeline(trained, proposal):
    # 32x32 torus, block schedule, guarded mixed precision: screening each
    # part of a stage on its own stream (overlapped pipeline) must give the
    # chain of the one-stream pipeline, visit for visit -- bit for bit at the
    # same CTA width; across widths the free energies differ by rounding, and
    # the decisions, screened visits and spins are the same.
    cfg = P.Config(Lx=32, Ly=32, L_c=8, schedule=P.SCHEDULE_BLOCK, T=0.05, mu=-6.5, seed=9, precision=P.MIXED,
                   proposal=proposal, cone_deg=30.0)
    runs = {}
    for pipe in (P.PIPELINE_STAGES, P.PIPELINE_OVERLAP):
        for w in (8, 4):
            ctx = P.Context(cfg)
            P.ptca_surrogate_set_params(ctx.h, trained["theta"], trained["scale"])
            P.ptca_surrogate_enable(ctx.h, True)
            P.ptca_set_launch_config(ctx.h, pipe, w)
            st = ctx.sweep(3)
            site, Fo, Fn, lnu, acc = ctx.record()
            runs[(pipe, w)] = (ctx.spins(), site, acc, Fo, Fn, (st.screened, st.eigensolves, st.accepted))
            ctx.close()
    ref = runs[(P.PIPELINE_STAGES, 8)]
    assert ref[5][0] > 0
    for key, r in runs.items():
        for a, b in zip(ref[:3], r[:3]):
            assert torch.equal(a, b), key
        assert r[5] == ref[5], key
        assert torch.equal(torch.isnan(r[3]), torch.isnan(ref[3]))
        ok = ~torch.isnan(ref[3])
        assert torch.max((r[3][ok] - ref[3][ok]).abs() / ref[3][ok].abs()).item() < 1e-5
    for w in (8, 4):
        a, b = runs[(P.PIPELINE_STAGES, w)], runs[(P.PIPELINE_OVERLAP, w)]
        for x, y in zip(a[3:5], b[3:5]):
            assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(y, nan=7.0)), w
    # Three one-sweep calls without statistics: each leaves its last re-solve
    # to the next call, and the next stage's screening and solves run beside
    # the current stage's (network buffers per stage parity).  Same chain.
    ctx = P.Context(cfg)
    P.ptca_surrogate_set_params(ctx.h, trained["theta"], trained["scale"])
    P.ptca_surrogate_enable(ctx.h, True)
    P.ptca_set_launch_config(ctx.h, P.PIPELINE_OVERLAP, 4)
    for _ in range(3):
        P.ptca_sweep(ctx.h, 1, stats=False)
    site, Fo, Fn, lnu, acc = ctx.record()
    ref4 = runs[(P.PIPELINE_STAGES, 4)]
    assert torch.equal(ctx.spins(), ref4[0]) and torch.equal(site, ref4[1]) and torch.equal(acc, ref4[2])
    for x, y in zip((Fo, Fn), ref4[3:5]):
        assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(y, nan=7.0))
    ctx.close()

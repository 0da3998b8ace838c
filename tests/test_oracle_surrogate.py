"""Pins of the FP64 reference surrogate network (oracle/surrogate.py)."""
import numpy as np
import pytest

from oracle import surrogate as S
from tests import inputs


def _theta(seed, scale=0.15):
    return inputs.rng(seed).normal(scale=scale, size=S.N_PARAMS)


def _feats(seed, n):
    spins = inputs.random_unit_spins(seed, n * 50).reshape(n, 50, 3)
    feat = np.concatenate([spins[:, :49, :].reshape(n, 147), spins[:, 49, :]], axis=1)
    center = inputs.rng(seed + 1).integers(0, 49, size=n)
    return feat, center


def test_bf16_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 3.0e-40, 65504.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0, 65536.0])
    got = S.bf16(vals)
    assert np.allclose(got[:5], want[:5], rtol=0, atol=0)
    assert abs(got[5]) < 1e-38  # subnormal range keeps its top bits; tiny either way
    assert got[6] == want[6]


def test_gradient_matches_central_differences():
    th = _theta(1)
    feat, center = _feats(2, 6)
    dF = inputs.rng(3).normal(size=6)
    loss, g = S.loss_and_grad(th, feat, center, dF, 0.7, rounding=False)
    rng = inputs.rng(4)
    idx = rng.choice(S.N_PARAMS, size=40, replace=False)
    # include biases and the last layer
    idx = np.concatenate([idx, [S.N_PARAMS - 8, S.N_PARAMS - 1 - 8 - 1, 256 * 160 + 3]])
    for i in idx:
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = S.loss_and_grad(tp, feat, center, dF, 0.7, rounding=False)
        lm, _ = S.loss_and_grad(tm, feat, center, dF, 0.7, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_surrogate_is_antisymmetric_under_swap():
    th = _theta(5)
    feat, center = _feats(6, 10)
    d = S.surrogate_dF(th, feat, center, 1.3)
    sw = feat.copy()
    for i in range(10):
        c = center[i]
        sw[i, 3 * c:3 * c + 3], sw[i, 147:150] = feat[i, 147:150], feat[i, 3 * c:3 * c + 3]
    assert np.allclose(S.surrogate_dF(th, sw, center, 1.3), -d, rtol=0, atol=1e-12)


def test_padding_does_not_change_h():
    th = _theta(7)
    feat, _ = _feats(8, 5)
    h0, _ = S.forward(th, feat)
    p = S.unpack(th)
    p["W1"][:, 150:] = 9.0
    p["W4"][1:, :] = -3.0
    p["b4"][1:] = 2.0
    h1, _ = S.forward(S.pack(p), feat)
    assert np.array_equal(h0, h1)


def test_canonical_frame_is_a_rotation_and_invariant():
    feat, center = _feats(9, 5)
    R = inputs.random_rotation(10)
    for i in range(5):
        c = center[i]
        x = S.canonical(feat[i].astype(np.float64), c)
        assert np.allclose(x[3 * c:3 * c + 3], [0, 0, 1], atol=1e-12)
        assert abs(x[148]) < 1e-12 and x[147] >= 0
        # norms preserved, and a global rotation of the input changes nothing
        assert np.allclose(np.linalg.norm(x.reshape(50, 3), axis=1), np.linalg.norm(feat[i].reshape(50, 3), axis=1))
        rot = (feat[i].reshape(50, 3) @ R.T).reshape(150)
        assert np.allclose(S.canonical(rot, c), x, atol=1e-12)

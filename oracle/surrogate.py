"""FP64 CPU reference of the surrogate network used for delayed acceptance.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the product never
imports it.  It defines what the GPU training and inference kernels compute,
written plainly with numpy:

  * h(x): 150 -> 256 -> 256 -> 256 -> 1 multilayer perceptron, SiLU
    activations (silu(z) = z / (1 + e^-z)) on the hidden layers, linear
    output.  The first layer's input is zero-padded from 150 to 160 and the
    last layer has 8 output rows of which only row 0 is used (tensor-core
    tile shapes); the padding never changes the value of h.
  * Every matrix product rounds both operands to bfloat16 (round to nearest,
    ties to even) and accumulates exactly (here in FP64; on the GPU in FP32).
    Biases, activations and the loss stay in full precision.
  * The surrogate of the free-energy change of a proposal s_old -> s_new at
    a site with environment patch P is
        dF~ = scale * ( h(c[P(s_old), s_new]) - h(c[P(s_new), s_old]) )
    which is antisymmetric under exchanging the two states, as delayed
    acceptance requires for detailed balance.  c[...] expresses a row in its
    own spin frame: the rotation taking the row's update-site spin a to +z and
    its last spin b into the xz half-plane with x >= 0 (e3 = a, e1 = the
    normalised part of b orthogonal to a -- or of x, or y, when b is parallel
    to a -- and e2 = e3 x e1).  The cluster spectrum is invariant under a
    global spin rotation, so the frame removes three symmetry directions.
  * Loss of a batch: mean over samples of (dF~/scale - dF/scale)^2.

Parameter vector layout (float32 on the GPU): W1[256x160], b1[256],
W2[256x256], b2[256], W3[256x256], b3[256], W4[8x256], b4[8].
"""
from __future__ import annotations

import numpy as np

D_IN, D_IN_PAD, D_H, D_OUT_PAD = 150, 160, 256, 8
SHAPES = [("W1", (D_H, D_IN_PAD)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)),
          ("W3", (D_H, D_H)), ("b3", (D_H,)), ("W4", (D_OUT_PAD, D_H)), ("b4", (D_OUT_PAD,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
PATCH = 7


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _mm(a, b, rounding):
    if rounding:
        a, b = bf16(a), bf16(b)
    return a @ b


def forward(theta, X, rounding=True):
    """h for rows of X (n x 150).  Returns (h, cache)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    A0 = np.zeros((X.shape[0], D_IN_PAD))
    A0[:, :D_IN] = X
    Z1 = _mm(A0, p["W1"].T, rounding) + p["b1"]
    A1 = silu(Z1)
    Z2 = _mm(A1, p["W2"].T, rounding) + p["b2"]
    A2 = silu(Z2)
    Z3 = _mm(A2, p["W3"].T, rounding) + p["b3"]
    A3 = silu(Z3)
    Z4 = _mm(A3, p["W4"].T, rounding) + p["b4"]
    return Z4[:, 0], (A0, Z1, A1, Z2, A2, Z3, A3)


def backward(theta, cache, dh, rounding=True):
    """Gradient of sum_i dh_i * h(x_i) with respect to the parameters."""
    p = unpack(theta)
    A0, Z1, A1, Z2, A2, Z3, A3 = cache
    g = {}
    dZ4 = np.zeros((dh.size, D_OUT_PAD))
    dZ4[:, 0] = dh
    g["W4"] = _mm(dZ4.T, A3, rounding)
    g["b4"] = dZ4.sum(axis=0)
    dZ3 = _mm(dZ4, p["W4"], rounding) * dsilu(Z3)
    g["W3"] = _mm(dZ3.T, A2, rounding)
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = _mm(dZ3, p["W3"], rounding) * dsilu(Z2)
    g["W2"] = _mm(dZ2.T, A1, rounding)
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = _mm(dZ2, p["W2"], rounding) * dsilu(Z1)
    g["W1"] = _mm(dZ1.T, A0, rounding)
    g["b1"] = dZ1.sum(axis=0)
    return pack(g)


def frame(a, b):
    """Rows e1, e2, e3 of the rotation that maps a to +z and b into the xz
    half-plane with x >= 0."""
    a = np.asarray(a, dtype=np.float64)
    a = a / np.linalg.norm(a)
    for cand in (np.asarray(b, dtype=np.float64), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])):
        r = cand - (cand @ a) * a
        nr = np.linalg.norm(r)
        if nr > 1e-6:
            e1 = r / nr
            break
    e2 = np.cross(a, e1)
    return np.vstack([e1, e2, a])


def canonical(row, c):
    """Row (150) in the frame of its update-site spin (entry c) and last spin."""
    R = frame(row[3 * c:3 * c + 3], row[147:150])
    return (row.reshape(50, 3) @ R.T).reshape(150)


def pair_inputs_with_center(feat, center):
    """Rows c[P(s_old), s_new] and c[P(s_new), s_old] from stored features
    (n x 150: the 7x7 patch, then s_new); center[i] is the patch index of the
    update site, whose entry holds s_old."""
    feat = np.asarray(feat, dtype=np.float64)
    n = feat.shape[0]
    x1 = feat.copy()
    x2 = feat.copy()
    for i in range(n):
        c = int(center[i])
        s_old = feat[i, 3 * c:3 * c + 3].copy()
        s_new = feat[i, 147:150].copy()
        x2[i, 3 * c:3 * c + 3] = s_new
        x2[i, 147:150] = s_old
        x1[i] = canonical(x1[i], c)
        x2[i] = canonical(x2[i], c)
    return x1, x2


def loss_and_grad(theta, feat, center, dF, scale, rounding=True):
    """Batch loss mean((h(x1) - h(x2) - dF/scale)^2) and its gradient."""
    x1, x2 = pair_inputs_with_center(feat, center)
    n = x1.shape[0]
    X = np.vstack([x1, x2])
    h, cache = forward(theta, X, rounding)
    r = h[:n] - h[n:] - np.asarray(dF, dtype=np.float64) / scale
    loss = float(np.mean(r * r))
    dh = np.concatenate([2.0 * r / n, -2.0 * r / n])
    return loss, backward(theta, cache, dh, rounding)


def surrogate_dF(theta, feat, center, scale, rounding=True):
    x1, x2 = pair_inputs_with_center(feat, center)
    h1, _ = forward(theta, x1, rounding)
    h2, _ = forward(theta, x2, rounding)
    return scale * (h1 - h2)

"""The learned radius proposer's network and features on the CPU (TEST
INFRASTRUCTURE ONLY: only tests/ use it).

The paper grows every sphere by sphere shrinking (Sec. 5.1) and has no
network; the library adds a multilayer perceptron that proposes where the
shrinking starts.  Written from the definitions, in fp64:

    h0 = relu(W0 x + b0), h1 = relu(W1 h0 + b1), h2 = relu(W2 h1 + b2),
    y = w3 . h2 + b3,  loss = mean over rows of (y - t)^2,

and its gradient by the chain rule, layer by layer from the output back:
dy = 2 (y - t) / n; for a layer z = W h + b feeding relu, dW = dz^T h,
db = sum of dz over rows, and the gradient reaching h is dz W masked by
h > 0 (the relu of the layer below).

With bf16=True the values are rounded to bfloat16 (round to nearest, ties to
even, of the float32 value) where the library stores them in that type: the
inputs, W0..W2, every hidden activation, and the hidden-layer gradients dz.
Everything else (w3, the biases, accumulations, the loss) stays wide.

Parameter vector layout (float32 in the library): W0[128][32], b0[128],
W1[128][128], b1[128], W2[128][128], b2[128], w3[128], b3.  Inputs narrower
than 32 use the first columns of W0.

Pins (tests/test_oracle_mlp.py): central finite differences of the fp64 loss,
the bfloat16 rounding against torch's conversion, the loss and gradient of a
network that fits its targets exactly (zero), and the features' identities.
"""
from __future__ import annotations

import numpy as np

HID, NIN = 128, 32
OW0 = 0
OB0 = OW0 + HID * NIN
OW1 = OB0 + HID
OB1 = OW1 + HID * HID
OW2 = OB1 + HID
OB2 = OW2 + HID * HID
OW3 = OB2 + HID
OB3 = OW3 + HID
NPARAM = OB3 + 1
N_FEATURES = 30


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) through float32; returns
    float64 values."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, n_in):
    p = np.asarray(p, dtype=np.float64)
    W0 = p[OW0:OB0].reshape(HID, NIN)[:, :n_in]
    return dict(W0=W0, b0=p[OB0:OW1], W1=p[OW1:OB1].reshape(HID, HID), b1=p[OB1:OW2],
                W2=p[OW2:OB2].reshape(HID, HID), b2=p[OB2:OW3], w3=p[OW3:OB3], b3=p[OB3])


def forward(p, x, bf=False):
    """Outputs y[n] and the activations (x, h0, h1, h2) as used."""
    x = np.asarray(x, dtype=np.float64)
    P = unpack(p, x.shape[1])
    r = bf16 if bf else (lambda a: a)
    X = r(x)
    H0 = r(np.maximum(X @ r(P["W0"]).T + P["b0"], 0.0))
    H1 = r(np.maximum(H0 @ r(P["W1"]).T + P["b1"], 0.0))
    H2 = r(np.maximum(H1 @ r(P["W2"]).T + P["b2"], 0.0))
    y = H2 @ P["w3"] + P["b3"]
    return y, (X, H0, H1, H2)


def loss(p, x, t, bf=False):
    y, _ = forward(p, x, bf)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, x, t, bf=False):
    """(gradient in the parameter layout, loss)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n, n_in = x.shape
    P = unpack(p, n_in)
    r = bf16 if bf else (lambda a: a)
    y, (X, H0, H1, H2) = forward(p, x, bf)
    g = np.zeros(NPARAM)
    dy = 2.0 * (y - t) / n
    g[OW3:OB3] = dy @ H2
    g[OB3] = dy.sum()
    dZ2 = r(np.outer(dy, P["w3"]) * (H2 > 0))
    g[OW2:OB2] = (dZ2.T @ H1).ravel()
    g[OB2:OW3] = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ r(P["W2"])) * (H1 > 0))
    g[OW1:OB1] = (dZ1.T @ H0).ravel()
    g[OB1:OW2] = dZ1.sum(axis=0)
    dZ0 = r((dZ1 @ r(P["W1"])) * (H0 > 0))
    gw0 = np.zeros((HID, NIN))
    gw0[:, :n_in] = dZ0.T @ X
    g[OW0:OB0] = gw0.ravel()
    g[OB0:OW1] = dZ0.sum(axis=0)
    return g, float(np.mean((y - t) ** 2))


def pin_features(pins, normals, lo, hi):
    """Proposer inputs of pins with unit inward normals in the box [lo, hi]:
    u = (p - centre) / (half the longest side), the normal, then
    sin(pi 2^o u_a) and cos(pi 2^o u_a) for o = 0..3, a = x, y, z."""
    pins = np.asarray(pins, dtype=np.float64)
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    centre = 0.5 * (lo + hi)
    half = 0.5 * float(np.max(hi - lo))
    u = (pins - centre) / half
    cols = [u, np.asarray(normals, dtype=np.float64)]
    for o in range(4):
        for a in range(3):
            cols.append(np.stack([np.sin(np.pi * 2 ** o * u[:, a]), np.cos(np.pi * 2 ** o * u[:, a])], axis=1))
    return np.concatenate(cols, axis=1)


def radius_target(radii, lo, hi):
    """log2(r / box diagonal)."""
    d = float(np.linalg.norm(np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)))
    return np.log2(np.asarray(radii, dtype=np.float64) / d)

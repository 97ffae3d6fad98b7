"""Oracle: the learned preconditioner T of the flexible CG and LOBPCG filters, in FP64.

Test infrastructure only (see ``oracle/__init__``).

The paper leaves the preconditioner T of Algorithms 2 and 3 open (Section 5 notes that
the flexible beta admits a variable, even nonlinear, T; Section 8 lists better
preconditioners as future work).  The learned T here is a small convolutional net applied
to the image-shaped residual r:

    c0 = (D^-1 r) / rho,  rho = rms(D^-1 r)       (the Jacobi-preconditioned residual)
    c1 = g                                           (the guide)
    c2 = 1 / d                                       (the inverse degree)
    A1 = conv(C, W1)   16 channels,  H1 = relu(A1)
    A2 = conv(H1, W2)  16 channels,  H2 = relu(A2)
    O  = conv(H2, W3)  1 channel
    T(r) = rho * O

Every conv is a 3 x 3 cross-correlation without bias; pixels outside the image contribute
zero.  T is positively homogeneous, T(c r) = c T(r) for c > 0, and with W1 carrying
+-c0 on two channels, W2 passing them through and W3 taking their difference it is
exactly Jacobi, T(r) = D^-1 r.

Training pairs (r, z) solve (L + sigma I) z = r; the loss of a pair is
||T(r) - z||^2 / ||z||^2.  ``backward`` returns its gradient with respect to W1, W2, W3
(rho depends on r only and is a constant for the weights).

Weights are arrays w[o][c][3][3] (output channel, input channel, tap row, tap column).
Pinned by tests/test_oracle_convnet.py: central finite differences of the loss, the
correlation against scipy.signal.correlate2d, the Jacobi special case and homogeneity.
"""
from __future__ import annotations

import numpy as np

CIN, CH = 3, 16
SHAPES = ((CH, CIN, 3, 3), (CH, CH, 3, 3), (1, CH, 3, 3))


def conv(x, w):
    """y[o, i, j] = sum_c sum_{a, b in -1..1} w[o, c, a+1, b+1] x[c, i+a, j+b] (zero outside)."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], H, W))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            shifted = xp[:, 1 + a:1 + a + H, 1 + b:1 + b + W]          # x[c, i+a, j+b]
            y += np.einsum("oc,chw->ohw", w[:, :, a + 1, b + 1], shifted)
    return y


def conv_t(g, w):
    """Adjoint of conv in its input: x[c, i, j] = sum_o sum_{a,b} w[o, c, a+1, b+1] g[o, i-a, j-b]."""
    O, H, W = g.shape
    gp = np.zeros((O, H + 2, W + 2))
    gp[:, 1:-1, 1:-1] = g
    x = np.zeros((w.shape[1], H, W))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            shifted = gp[:, 1 - a:1 - a + H, 1 - b:1 - b + W]          # g[o, i-a, j-b]
            x += np.einsum("oc,ohw->chw", w[:, :, a + 1, b + 1], shifted)
    return x


def conv_wgrad(g, x):
    """dW[o, c, a+1, b+1] = sum_{i,j} g[o, i, j] x[c, i+a, j+b] (gradient of <g, conv(x, W)>)."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros((g.shape[0], C, 3, 3))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            dw[:, :, a + 1, b + 1] = np.einsum("ohw,chw->oc", g, xp[:, 1 + a:1 + a + H, 1 + b:1 + b + W])
    return dw


def inputs(r, guide, d):
    """The three input channels and rho for a residual image r (H x W)."""
    c0 = np.asarray(r, np.float64) / np.asarray(d, np.float64)
    rho = float(np.sqrt(np.mean(c0 * c0)))
    C = np.stack([c0 / rho if rho > 0 else np.zeros_like(c0),
                  np.asarray(guide, np.float64), 1.0 / np.asarray(d, np.float64)])
    return C, rho


def forward(r, guide, d, W):
    """T(r) and the intermediates (C, rho, A1, A2, O)."""
    W1, W2, W3 = W
    C, rho = inputs(r, guide, d)
    A1 = conv(C, W1)
    A2 = conv(np.maximum(A1, 0.0), W2)
    O = conv(np.maximum(A2, 0.0), W3)
    return rho * O[0], dict(C=C, rho=rho, A1=A1, A2=A2, O=O)


def loss(r, guide, d, z, W):
    T, _ = forward(r, guide, d, W)
    return float(np.sum((T - z) ** 2) / np.sum(np.asarray(z, np.float64) ** 2))


def backward(r, guide, d, z, W):
    """(loss, [dW1, dW2, dW3]) for one pair."""
    W1, W2, W3 = W
    T, c = forward(r, guide, d, W)
    z = np.asarray(z, np.float64)
    zz = float(np.sum(z * z))
    L = float(np.sum((T - z) ** 2) / zz)
    G3 = (2.0 * c["rho"] / zz * (T - z))[None]            # dL/dO
    H2 = np.maximum(c["A2"], 0.0)
    H1 = np.maximum(c["A1"], 0.0)
    dW3 = conv_wgrad(G3, H2)
    G2 = conv_t(G3, W3) * (c["A2"] > 0)
    dW2 = conv_wgrad(G2, H1)
    G1 = conv_t(G2, W2) * (c["A1"] > 0)
    dW1 = conv_wgrad(G1, c["C"])
    return L, [dW1, dW2, dW3]


def jacobi_weights(noise: float = 0.0, seed: int = 0):
    """Weights with which T is exactly D^-1 when noise = 0: channels 0 and 1 of layer 1 carry
    +c0 and -c0, layer 2 passes them through, layer 3 takes their difference.  With
    noise > 0 every other weight is N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    W1, W2, W3 = [noise * rng.standard_normal(s) for s in SHAPES]
    W1[0:2] = 0.0
    W1[0, 0, 1, 1] = 1.0
    W1[1, 0, 1, 1] = -1.0
    W2[0:2] = 0.0
    W2[0, 0, 1, 1] = 1.0
    W2[1, 1, 1, 1] = 1.0
    W3[0, 0:2] = 0.0
    W3[0, 0, 1, 1] = 1.0
    W3[0, 1, 1, 1] = -1.0
    return [W1, W2, W3]


def adam_step(W, G, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) of the weight list W with gradients G, moments m, v
    and step number t >= 1; returns the new (W, m, v)."""
    Wn, mn, vn = [], [], []
    for w, g, mm, vv in zip(W, G, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        Wn.append(w - lr * mh / (np.sqrt(vh) + eps))
        mn.append(mm)
        vn.append(vv)
    return Wn, mn, vn

"""Oracle: a learned symmetric positive definite preconditioner T, in FP64.

Test infrastructure only (see ``oracle/__init__``).

The paper leaves the preconditioner T of Algorithms 2 and 3 open (Section 5; Section 8
names better preconditioners as future work).  CG keeps the optimality of Section 5 -- the
iterate minimises the A-norm of the error over the Krylov space -- when T is symmetric
and positive definite, and the Ritz vectors of LOBPCG (Algorithm 3) need a linear T.  The
T here is linear, symmetric and positive definite by construction:

    T r = D^-1/2 (u + K^T K u),      u = D^-1/2 r,

where K is a (2h + 1) x (2h + 1) cross-correlation of the image-shaped u (pixels outside
the image contribute zero) and K^T is its adjoint: the correlation with the kernel turned
by 180 degrees, again with zeros outside.  With K = 0 it is Jacobi, T = D^-1.

Training pairs (r, z) solve A z = r with A = L + sigma I.  The loss of a pair measures T r
as an approximation of z in the A-norm, relative to z:

    loss = (z - T r)^T A (z - T r) / (z^T A z).

``loss_grad`` returns it with its gradient with respect to K.  Pinned by
tests/test_oracle_precond_spd.py: the correlation against scipy.signal.correlate2d, the
adjoint identity, symmetry and positive definiteness of T, the Jacobi special case,
central finite differences of the loss, and the A-norm optimality of CG with this T.
"""
from __future__ import annotations

import numpy as np


def correlate(x, K):
    """y[i, j] = sum_{a, b in -h..h} K[a + h, b + h] x[i + a, j + b], zero outside the
    image (x: (ny, nx), K: (2h + 1, 2h + 1))."""
    x = np.asarray(x, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    h = K.shape[0] // 2
    ny, nx = x.shape
    y = np.zeros_like(x)
    for a in range(-h, h + 1):
        for b in range(-h, h + 1):
            # output rows i with 0 <= i + a < ny, columns j with 0 <= j + b < nx
            i0, i1 = max(0, -a), min(ny, ny - a)
            j0, j1 = max(0, -b), min(nx, nx - b)
            if i0 >= i1 or j0 >= j1:
                continue
            y[i0:i1, j0:j1] += K[a + h, b + h] * x[i0 + a:i1 + a, j0 + b:j1 + b]
    return y


def correlate_adjoint(y, K):
    """The adjoint of ``correlate`` for the same K: the correlation with K turned by 180
    degrees (x[i, j] = sum K[a + h, b + h] y[i - a, j - b], zero outside)."""
    return correlate(y, np.asarray(K)[::-1, ::-1])


def apply(K, d, shape, r):
    """T r for r of n = ny * nx entries, or a block [n][k] (T applied to each column)."""
    r = np.asarray(r, dtype=np.float64)
    dh = 1.0 / np.sqrt(np.asarray(d, dtype=np.float64))
    if r.ndim == 2:
        return np.stack([apply(K, d, shape, r[:, c]) for c in range(r.shape[1])], axis=1)
    u = (dh * r).reshape(shape)
    t = u + correlate_adjoint(correlate(u, K), K)
    return dh * t.reshape(-1)


def matrix(K, d, shape):
    """T as a dense matrix (tiny images only): its columns are T e_j."""
    n = shape[0] * shape[1]
    return np.stack([apply(K, d, shape, np.eye(n)[:, j]) for j in range(n)], axis=1)


def loss_grad(K, d, shape, A, r, z):
    """(loss, dloss/dK) of one pair (r, z) with A z = r; A is a sparse or dense n x n
    matrix.  With u = D^-1/2 r, w = K u, t = D^-1/2 (u + K^T w), e = z - t and
    h = D^-1/2 dloss/dt = -2 D^-1/2 A e / (z^T A z):
        dloss/dK[a, b] = sum_p w(p) h(p + (a, b)) + sum_p (K h)(p) u(p + (a, b)),
    zero-padded at the border."""
    K = np.asarray(K, dtype=np.float64)
    hk = K.shape[0] // 2
    dh = 1.0 / np.sqrt(np.asarray(d, dtype=np.float64))
    r = np.asarray(r, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    u = (dh * r).reshape(shape)
    w = correlate(u, K)
    t = dh * (u + correlate_adjoint(w, K)).reshape(-1)
    e = z - t
    Ae = A @ e
    c = float(z @ (A @ z))
    loss = float(e @ Ae) / c
    hv = (dh * (-2.0 * Ae / c)).reshape(shape)
    kh = correlate(hv, K)
    ny, nx = shape
    grad = np.zeros_like(K)
    for a in range(-hk, hk + 1):
        for b in range(-hk, hk + 1):
            i0, i1 = max(0, -a), min(ny, ny - a)
            j0, j1 = max(0, -b), min(nx, nx - b)
            if i0 >= i1 or j0 >= j1:
                continue
            s1 = np.sum(w[i0:i1, j0:j1] * hv[i0 + a:i1 + a, j0 + b:j1 + b])
            s2 = np.sum(kh[i0:i1, j0:j1] * u[i0 + a:i1 + a, j0 + b:j1 + b])
            grad[a + hk, b + hk] = s1 + s2
    return loss, grad


def identity_kernel(half: int, scale: float = 0.0):
    """K = scale * delta (the centre tap): T = (1 + scale^2) D^-1; scale 0 gives Jacobi."""
    K = np.zeros((2 * half + 1, 2 * half + 1))
    K[half, half] = scale
    return K

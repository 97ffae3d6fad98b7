"""Oracle: the guided filter of Section 3 as a vector transform (Algorithm 1, Eqs. 5-6).

Test infrastructure only (see ``oracle/__init__``).

* ``box_mean``       -- the mean filter f_mean of Algorithm 1 over a square window of
                        radius r (width rho = 2r + 1; 1D: an interval), truncated at the
                        border: each pixel averages the in-image pixels of its window.
* ``guided_filter``  -- Algorithm 1 step by step: mean_g, mean_x, corr_g, corr_gx, var_g,
                        cov_gx, a, b, mean_a, mean_b, y = mean_a .* g + mean_b.
* ``GuidedGraph``    -- the matrix of Eq. 6 built entry by entry from the windows, its
                        degree and Laplacian, as explicit FP64 CSR matrices.

Reading of the border (the paper takes |omega| equal for all windows, i.e. no border).
With truncated windows, window omega_k holds N_k in-image pixels, and mu_k, sigma_k^2 are
the mean and variance over them.  The symmetric matrix
    Wt_ij = sum_{k : i, j in omega_k} (1 / N_k) (1 + (g_i - mu_k)(g_j - mu_k) / (sigma_k^2 + eps))
has row sums N_i (the number of windows that contain i, which for a square window equals
the number of in-image pixels of the window centred at i), so D = diag(N), L = D - Wt is
the graph Laplacian, and Algorithm 1 with truncated mean filters computes exactly
y = D^-1 Wt x.  Away from the border N = |omega| and Wt / |omega| is Eq. 6 (whose rows sum
to 1, D = I in the paper's normalisation): the pencil (L, D) is the paper's (I - W, I)
scaled by |omega|.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _offsets(ndim: int, r: int):
    dys = range(-r, r + 1) if ndim == 2 else [0]
    return [(dy, dx) for dy in dys for dx in range(-r, r + 1)]


def box_mean(v, shape, r: int):
    """f_mean(v, 2r + 1): mean over the in-image pixels of each pixel's window."""
    ny, nx = shape
    V = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    ndim = 1 if ny == 1 else 2
    acc = np.zeros_like(V)
    cnt = np.zeros_like(V)
    for dy, dx in _offsets(ndim, r):
        ys0, ys1 = max(0, -dy), min(ny, ny - dy)
        xs0, xs1 = max(0, -dx), min(nx, nx - dx)
        acc[ys0:ys1, xs0:xs1] += V[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
        cnt[ys0:ys1, xs0:xs1] += 1.0
    return (acc / cnt).reshape(-1)


def window_count(shape, r: int):
    """N_i: in-image pixels of the window centred at i."""
    return _count(shape, r)


def _count(shape, r):
    ny, nx = shape
    ndim = 1 if ny == 1 else 2
    cnt = np.zeros((ny, nx))
    for dy, dx in _offsets(ndim, r):
        ys0, ys1 = max(0, -dy), min(ny, ny - dy)
        xs0, xs1 = max(0, -dx), min(nx, nx - dx)
        cnt[ys0:ys1, xs0:xs1] += 1.0
    return cnt.reshape(-1)


def guided_filter(x, g, shape, r: int, eps: float):
    """Algorithm 1 (guided filter) with f_mean = box_mean of radius r."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    mean_g = box_mean(g, shape, r)
    mean_x = box_mean(x, shape, r)
    corr_g = box_mean(g * g, shape, r)
    corr_gx = box_mean(g * x, shape, r)
    var_g = corr_g - mean_g * mean_g
    cov_gx = corr_gx - mean_g * mean_x
    a = cov_gx / (var_g + eps)
    b = mean_x - a * mean_g
    mean_a = box_mean(a, shape, r)
    mean_b = box_mean(b, shape, r)
    return mean_a * g + mean_b


class GuidedGraph:
    """Wt of Eq. 6 (border reading above), D = diag(N), L = D - Wt, D^-1 Wt, as CSR."""

    def __init__(self, guide, shape, r: int, eps: float):
        ny, nx = shape
        self.shape = (ny, nx)
        self.n = n = ny * nx
        self.r, self.eps = r, eps
        ndim = 1 if ny == 1 else 2
        g = np.asarray(guide, dtype=np.float64).reshape(-1)
        self.guide = g.copy()
        rows, cols, vals = [], [], []
        for ky in range(ny):
            for kx in range(nx):
                members = [(ky + dy) * nx + (kx + dx) for dy, dx in _offsets(ndim, r)
                           if 0 <= ky + dy < ny and 0 <= kx + dx < nx]
                m = np.array(members)
                gk = g[m]
                nk = len(m)
                mu = gk.mean()
                var = ((gk - mu) ** 2).mean()
                dev = gk - mu
                block = (1.0 + np.outer(dev, dev) / (var + eps)) / nk
                rows.append(np.repeat(m, nk))
                cols.append(np.tile(m, nk))
                vals.append(block.reshape(-1))
        self.W = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(n, n))
        self.W.sum_duplicates()
        self.d = np.asarray(self.W.sum(axis=1)).reshape(-1)
        self.N = _count(shape, r)
        self.D = sp.diags(self.d).tocsr()
        self.L = (self.D - self.W).tocsr()
        self.DINV_W = (sp.diags(1.0 / self.d) @ self.W).tocsr()

"""Oracle: the guided filter of Section 3 as a vector transform (Algorithm 1, Eqs. 5-6).

Test infrastructure only (see ``oracle/__init__``).

* ``box_mean``       -- the mean filter f_mean of Algorithm 1 over a square window of
                        radius r (width rho = 2r + 1; 1D: an interval), truncated at the
                        border: each pixel averages the in-image pixels of its window.
* ``guided_filter``  -- the transform Algorithm 1 computes, from its definition (Section 3,
                        Eqs. 5-6): in every window the signal is fitted by a line in the
                        guide, x ~ a_k g + b_k, by least squares with a ridge eps * a_k^2 per
                        window pixel; the output at a pixel is the mean of the predictions
                        a_k g_i + b_k of all windows that contain it.
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


def _window_sums(v, shape, r: int):
    """(sum of v over the in-image pixels of each pixel's window, number of those pixels).
    For square windows pixel j lies in the window centred at i exactly when i lies in the
    window centred at j, so the same sums run over the windows that contain a pixel."""
    ny, nx = shape
    V = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    total = np.zeros_like(V)
    count = np.zeros_like(V)
    for dy, dx in _offsets(1 if ny == 1 else 2, r):
        y0, y1 = max(0, -dy), min(ny, ny - dy)
        x0, x1 = max(0, -dx), min(nx, nx - dx)
        total[y0:y1, x0:x1] += V[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        count[y0:y1, x0:x1] += 1.0
    return total.reshape(-1), count.reshape(-1)


def guided_filter(x, g, shape, r: int, eps: float):
    """The guided filter of Section 3 (what Algorithm 1 computes with f_mean = box_mean of
    radius r), from its definition.

    Window k (centred at pixel k, N_k in-image pixels) fits the line a_k g + b_k to x by
    minimising  sum_{j in window k} ((a_k g_j + b_k - x_j)^2 + eps a_k^2).  Setting the two
    partial derivatives to zero gives the normal equations
        (G2 + N eps) a + G1 b = GX,     G1 a + N b = X1,
    with G1 = sum g_j, G2 = sum g_j^2, X1 = sum x_j, GX = sum g_j x_j over the window; they
    are solved by Cramer's rule.  Pixel i then takes the mean over the windows k that
    contain it of the prediction a_k g_i + b_k."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    G1, N = _window_sums(g, shape, r)
    G2, _ = _window_sums(g * g, shape, r)
    X1, _ = _window_sums(x, shape, r)
    GX, _ = _window_sums(g * x, shape, r)
    m11 = G2 + N * eps                       # the 2 x 2 system [[m11, G1], [G1, N]]
    det = m11 * N - G1 * G1
    slope = (GX * N - G1 * X1) / det
    icpt = (m11 * X1 - G1 * GX) / det
    slope_sum, nwin = _window_sums(slope, shape, r)
    icpt_sum, _ = _window_sums(icpt, shape, r)
    return (slope_sum * g + icpt_sum) / nwin


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

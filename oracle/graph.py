"""Oracle: the bilateral-filter graph as explicit FP64 sparse matrices.

Test infrastructure only (see ``oracle/__init__``).

Section 2: the weight between pixels i and j is (Eq. 2)

    w_ij = exp(-|p_i - p_j|^2 / (2 sigma_s^2)) * exp(-|g_i - g_j|^2 / (2 sigma_r^2))

for j in the window around i, where g is the guide (the noisy signal itself when
self-guided).  W = (w_ij) is symmetric with w_ij >= 0, D = diag(d) with d_i = sum_j w_ij,
the BF step is y = D^-1 W x (Eq. 3) and L = D - W (Eq. 4).  Section 4 adds the normalised
Laplacian (diag L)^-1/2 L (diag L)^-1/2.

Readings of the text where it leaves a choice, each with its reason:
* the sum in Eq. 1 runs over all j of the window, j = i included, and Eq. 2 gives that
  term exp(0) exp(0) = 1, so w_ii = 1 is part of W and of d_i (it cancels in L);
* the window is square (Chebyshev radius r, |dx| <= r and |dy| <= r), since the paper
  sizes it by one width in both directions, or, for the 5-point lattice of the Section 7
  image experiment, a cross (dx = 0 or dy = 0); the graph's vertices are the pixels, so
  neighbours that fall outside the image do not exist (no padding);
* |p_i - p_j| in Eq. 2 is the distance between pixel positions: Euclidean in grid units
  (the sample index in 1D);
* besides the paper's (diag L)-normalised Laplacian ("NDIAGL") the oracle also builds
  D^-1/2 L D^-1/2 ("NSYM"), whose spectrum is that of the pencil (L, D) used by CG and
  LOBPCG.  A pixel with diag L = 0 (no neighbour of positive weight) gets a zero row and
  column in NDIAGL.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

OPS = ("W", "L", "DINV_W", "D", "NSYM", "NDIAGL")


def window_offsets(ndim: int, radius: int, window: str = "square"):
    """Window taps (dy, dx), row-major: dy from -r to r, then dx from -r to r.

    The order is the canonical tap order used when weights are exported per tap."""
    out = []
    dys = range(-radius, radius + 1) if ndim == 2 else [0]
    for dy in dys:
        for dx in range(-radius, radius + 1):
            if window == "cross" and dx != 0 and dy != 0:
                continue
            out.append((dy, dx))
    return out


def spatial_factor(dy: int, dx: int, sigma_s: float) -> float:
    """First factor of Eq. 2 (np.inf for sigma_s switches it off)."""
    return float(np.exp(-(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s)))


class Graph:
    """Explicit W, D, L of Eqs. 2-4 for a 1D signal (ny = 1) or a 2D image (ny, nx)."""

    def __init__(self, guide, shape, radius: int, sigma_s: float, sigma_r: float,
                 window: str = "square"):
        ny, nx = shape
        self.shape = (ny, nx)
        self.ndim = 1 if ny == 1 else 2
        self.n = n = ny * nx
        self.radius, self.sigma_s, self.sigma_r, self.window = radius, sigma_s, sigma_r, window
        g = np.asarray(guide, dtype=np.float64).reshape(ny, nx)
        self.guide = g.reshape(-1).copy()
        self.offsets = window_offsets(self.ndim, radius, window)
        yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        rows, cols, vals = [], [], []
        # taps[t][i] = w(i, i + offset_t), 0 where the neighbour does not exist
        self.taps = np.zeros((n, len(self.offsets)), dtype=np.float64)
        for t, (dy, dx) in enumerate(self.offsets):
            ty, tx = yy + dy, xx + dx
            ok = (ty >= 0) & (ty < ny) & (tx >= 0) & (tx < nx)
            i = (yy * nx + xx)[ok]
            j = (ty * nx + tx)[ok]
            gi = g[yy[ok], xx[ok]]
            gj = g[ty[ok], tx[ok]]
            w = spatial_factor(dy, dx, sigma_s) * np.exp(-((gi - gj) ** 2) / (2.0 * sigma_r * sigma_r))
            rows.append(i)
            cols.append(j)
            vals.append(w)
            self.taps[i, t] = w
        self._assemble(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))

    @classmethod
    def from_taps(cls, taps, shape, radius: int, window: str = "square"):
        """The graph whose weights are given per tap: taps[i, t] = w(i, i + offset_t) in
        the canonical tap order (entries for neighbours outside the image are ignored).
        Used to build the exact FP64 operator of weights that were rounded for storage."""
        ny, nx = shape
        self = cls.__new__(cls)
        self.shape = (ny, nx)
        self.ndim = 1 if ny == 1 else 2
        self.n = n = ny * nx
        self.radius, self.sigma_s, self.sigma_r, self.window = radius, None, None, window
        self.guide = None
        self.offsets = window_offsets(self.ndim, radius, window)
        taps = np.asarray(taps, dtype=np.float64).reshape(n, len(self.offsets))
        yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        rows, cols, vals = [], [], []
        self.taps = np.zeros((n, len(self.offsets)), dtype=np.float64)
        for t, (dy, dx) in enumerate(self.offsets):
            ty, tx = yy + dy, xx + dx
            ok = (ty >= 0) & (ty < ny) & (tx >= 0) & (tx < nx)
            i = (yy * nx + xx)[ok]
            j = (ty * nx + tx)[ok]
            w = taps[i, t]
            rows.append(i)
            cols.append(j)
            vals.append(w)
            self.taps[i, t] = w
        self._assemble(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
        return self

    def _assemble(self, rows, cols, vals):
        n = self.n
        self.W = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
        self.d = np.asarray(self.W.sum(axis=1)).reshape(-1)        # d_i = sum_j w_ij
        self.D = sp.diags(self.d)
        self.L = (self.D - self.W).tocsr()                          # Eq. 4
        # diag L_i = sum_{j != i} w_ij, taken from the off-diagonal entries themselves
        off = rows != cols
        self.diagL = np.bincount(rows[off], weights=vals[off], minlength=n)
        dis = 1.0 / np.sqrt(self.d)
        self.NSYM = (sp.diags(dis) @ self.L @ sp.diags(dis)).tocsr()
        ok = self.diagL > 1e-30
        dls = np.zeros(n)
        dls[ok] = 1.0 / np.sqrt(self.diagL[ok])
        self.NDIAGL = (sp.diags(dls) @ self.L @ sp.diags(dls)).tocsr()
        self.DINV_W = (sp.diags(1.0 / self.d) @ self.W).tocsr()     # Eq. 3

    def matrix(self, op: str):
        return {"W": self.W, "L": self.L, "DINV_W": self.DINV_W, "D": self.D.tocsr(),
                "NSYM": self.NSYM, "NDIAGL": self.NDIAGL}[op]

    def apply(self, op: str, X):
        """op . X for X of shape [n] or [n][k] (pixel-major)."""
        X = np.asarray(X, dtype=np.float64)
        return np.asarray(self.matrix(op) @ X)

    def dense(self, op: str = "L"):
        return self.matrix(op).toarray()

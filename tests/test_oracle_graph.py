"""Pins of the oracle's graph (Section 2, Eqs. 1-4; Section 4) against facts the paper and
the mathematics fix -- never against the CUDA path."""
import json
import math
import os

import numpy as np
import pytest
import scipy.signal

from oracle.graph import Graph, window_offsets
from paper_1509_02468_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_graph(ndim, seed=0, n=37, ny=9, nx=11, radius=2, ss=1.5, sr=0.2, window="square"):
    rng = np.random.default_rng(seed)
    if ndim == 1:
        g = rng.uniform(0, 1, n)
        return Graph(g, (1, n), radius, ss, sr, window)
    g = rng.uniform(0, 1, (ny, nx))
    return Graph(g, (ny, nx), radius, ss, sr, window)


def test_hand_computed_tiny_1d():
    """Eq. 2 with numbers worked by hand (golden fixture)."""
    fx = json.load(open(os.path.join(GOLDEN, "tiny1d_weights.json")))
    G = Graph(np.array(fx["guide"]), (1, 3), fx["radius"], fx["sigma_s"], fx["sigma_r"])
    np.testing.assert_allclose(G.W.toarray(), np.array(fx["W"]), rtol=1e-14, atol=0)
    np.testing.assert_allclose(G.d, np.array(fx["d"]), rtol=1e-14)
    np.testing.assert_allclose(G.L.toarray(), np.array(fx["L"]), rtol=1e-14, atol=1e-16)


def test_window_shapes():
    assert len(window_offsets(1, 5)) == 11
    assert len(window_offsets(2, 3)) == 49
    assert window_offsets(2, 1, "cross") == [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    # tap order is row-major in (dy, dx)
    offs = window_offsets(2, 2)
    assert offs == sorted(offs)


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("window", ["square", "cross"])
def test_symmetric_nonnegative_unit_diagonal(ndim, window):
    """P1: W = W^T, w_ij in (0, 1], w_ii = 1 (Section 2: W symmetric, w_ij >= 0)."""
    G = _rand_graph(ndim, window=window)
    W = G.W.toarray()
    assert np.array_equal(W, W.T)
    nz = W[W != 0]
    assert nz.min() > 0 and nz.max() <= 1.0
    assert np.all(np.diag(W) == 1.0)


@pytest.mark.parametrize("ndim", [1, 2])
def test_bf_step_rows_sum_to_one(ndim):
    """P2: D^-1 W is an averaging operator (Eq. 1): its rows sum to 1."""
    G = _rand_graph(ndim, seed=1)
    np.testing.assert_allclose(G.DINV_W @ np.ones(G.n), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(G.apply("DINV_W", np.ones(G.n)), 1.0, atol=1e-15)


@pytest.mark.parametrize("ndim", [1, 2])
def test_laplacian_null_vector_and_psd(ndim):
    """P3: L e = 0 and L is symmetric non-negative definite (Section 4)."""
    G = _rand_graph(ndim, seed=2)
    np.testing.assert_allclose(G.L @ np.ones(G.n), 0.0, atol=1e-14)
    lam = np.linalg.eigvalsh(G.dense("L"))
    assert lam.min() > -1e-12


@pytest.mark.parametrize("ndim", [1, 2])
def test_normalised_spectra(ndim):
    """P4: spec(D^-1/2 L D^-1/2) in [0, 2) and spec((diag L)^-1/2 L (diag L)^-1/2) in [0, 2]."""
    G = _rand_graph(ndim, seed=3)
    a = np.linalg.eigvalsh(G.dense("NSYM"))
    b = np.linalg.eigvalsh(G.dense("NDIAGL"))
    assert a.min() > -1e-12 and a.max() < 2.0
    assert b.min() > -1e-12 and b.max() <= 2.0 + 1e-12
    # NDIAGL has unit diagonal (its diagonal is diag L / diag L)
    np.testing.assert_allclose(np.diag(G.dense("NDIAGL")), 1.0, atol=1e-14)
    # D^-1/2 L D^-1/2 is similar to D^-1 L: same spectrum as the pencil (L, D), and its
    # null vector is D^1/2 e
    import scipy.linalg as sla
    ref = sla.eigh(G.dense("L"), np.diag(G.d), eigvals_only=True)
    np.testing.assert_allclose(np.sort(a), np.sort(ref), atol=1e-12)
    np.testing.assert_allclose(G.apply("NSYM", np.sqrt(G.d)), 0.0, atol=1e-14)
    np.testing.assert_allclose(G.apply("NDIAGL", np.sqrt(G.diagL)), 0.0, atol=1e-14)


def test_isolated_pixel_ndiagl_row_is_zero():
    """A pixel whose neighbours all have weight 0 (underflow) has diag L = 0: NDIAGL row = 0."""
    g = np.array([0.0, 0.0, 100.0, 0.0])
    G = Graph(g, (1, 4), 1, 1.0, 0.01)
    assert G.diagL[2] == 0.0
    M = G.dense("NDIAGL")
    assert np.all(M[2] == 0) and np.all(M[:, 2] == 0)


def test_path_laplacian_closed_form():
    """P5: sigma_s = sigma_r = inf and r = 1 in 1D give the path graph Laplacian, whose
    eigenvalues are 2 - 2 cos(pi j / n)."""
    n = 40
    G = Graph(np.random.default_rng(0).uniform(size=n), (1, n), 1, np.inf, np.inf)
    lam = np.linalg.eigvalsh(G.dense("L"))
    ref = 2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n)
    np.testing.assert_allclose(np.sort(lam), np.sort(ref), atol=1e-12)


def test_grid_laplacian_closed_form_cross():
    """P5: the 5-point lattice (Section 7) with infinite sigmas is the grid Laplacian
    L1 (x) I + I (x) L1; its eigenvalues are sums of two path eigenvalues."""
    ny, nx = 7, 9
    G = Graph(np.zeros((ny, nx)), (ny, nx), 1, np.inf, np.inf, window="cross")
    lam = np.sort(np.linalg.eigvalsh(G.dense("L")))
    lx = 2.0 - 2.0 * np.cos(np.pi * np.arange(nx) / nx)
    ly = 2.0 - 2.0 * np.cos(np.pi * np.arange(ny) / ny)
    ref = np.sort((ly[:, None] + lx[None, :]).reshape(-1))
    np.testing.assert_allclose(lam, ref, atol=1e-12)


def test_square_window_kronecker_pencil():
    """P5: with infinite sigmas the square window is a Kronecker product W = A_y (x) A_x,
    D = D_y (x) D_x, so the pencil (L, D) of the image has eigenvalues
    1 - (1 - a)(1 - b) with a, b eigenvalues of the 1D pencils (catches 2D indexing)."""
    ny, nx, r = 6, 8, 2
    G = Graph(np.zeros((ny, nx)), (ny, nx), r, np.inf, np.inf)
    Gy = Graph(np.zeros(ny), (1, ny), r, np.inf, np.inf)
    Gx = Graph(np.zeros(nx), (1, nx), r, np.inf, np.inf)
    import scipy.linalg as sla
    lam = np.sort(sla.eigh(G.dense("L"), np.diag(G.d), eigvals_only=True))
    a = sla.eigh(Gy.dense("L"), np.diag(Gy.d), eigvals_only=True)
    b = sla.eigh(Gx.dense("L"), np.diag(Gx.d), eigvals_only=True)
    ref = np.sort((1.0 - (1.0 - a[:, None]) * (1.0 - b[None, :])).reshape(-1))
    np.testing.assert_allclose(lam, ref, atol=1e-12)


def test_range_off_is_normalised_gaussian_convolution_1d():
    """P5: with sigma_r = inf, away from the ends, one BF step D^-1 W x is a direct
    convolution with the Gaussian exp(-t^2 / (2 sigma_s^2)), t = -r..r, normalised to 1."""
    n, r, ss = 64, 4, 1.7
    x = np.random.default_rng(5).standard_normal(n)
    G = Graph(x, (1, n), r, ss, np.inf)
    t = np.arange(-r, r + 1)
    kern = np.exp(-t ** 2 / (2 * ss * ss))
    ref = np.convolve(x, kern / kern.sum(), mode="same")
    y = G.apply("DINV_W", x)
    np.testing.assert_allclose(y[r:-r], ref[r:-r], rtol=1e-13, atol=1e-13)


def test_range_off_is_normalised_gaussian_convolution_2d():
    """As above for the 7x7 window of the image configuration (scipy convolve2d)."""
    ny, nx, r, ss = 20, 23, 3, 2.0
    x = np.random.default_rng(6).standard_normal((ny, nx))
    G = Graph(x, (ny, nx), r, ss, np.inf)
    t = np.arange(-r, r + 1)
    k1 = np.exp(-t ** 2 / (2 * ss * ss))
    kern = np.outer(k1, k1)
    ref = scipy.signal.convolve2d(x, kern / kern.sum(), mode="same")
    y = G.apply("DINV_W", x.reshape(-1)).reshape(ny, nx)
    np.testing.assert_allclose(y[r:-r, r:-r], ref[r:-r, r:-r], rtol=1e-12, atol=1e-13)


def test_range_factor_two_pixels():
    """Eq. 2's range factor alone: two pixels, sigma_s = inf: w01 = exp(-(g0-g1)^2/(2 s_r^2))."""
    for g1, sr in [(0.3, 0.1), (0.05, 0.08), (1.0, 2.0)]:
        G = Graph(np.array([0.0, g1]), (1, 2), 1, np.inf, sr)
        assert math.isclose(G.W[0, 1], math.exp(-g1 * g1 / (2 * sr * sr)), rel_tol=1e-15)


def test_taps_match_matrix():
    """The per-tap export taps[i, t] = w(i, i + offset_t) (0 off the image)."""
    G = _rand_graph(2, seed=7, ny=5, nx=6, radius=1)
    W = G.W.toarray()
    ny, nx = G.shape
    for i in range(G.n):
        y, x = divmod(i, nx)
        for t, (dy, dx) in enumerate(G.offsets):
            yy, xx = y + dy, x + dx
            exp = W[i, yy * nx + xx] if (0 <= yy < ny and 0 <= xx < nx) else 0.0
            assert G.taps[i, t] == exp


def test_gershgorin_smoothing_bound():
    """Section 2: max_i d_i <= 2 makes the step x - L x smoothing.  By Gershgorin every
    eigenvalue of L lies in [0, 2 (d_i - 1)] (w_ii = 1 included), so ||I - L|| <= 1."""
    g = np.repeat(np.array([0.0, 1.0, 0.0, 1.0]), 5)
    G = Graph(g, (1, g.size), 1, 0.5, 0.05)
    assert G.d.max() <= 2.0
    lam = np.linalg.eigvalsh(np.eye(G.n) - G.dense("L"))
    assert np.abs(lam).max() <= 1.0 + 1e-12


def test_synthetic_noise_psnr_matches_paper_caption():
    """Section 7: noise variance 0.01 gives PSNR about 20.1 dB; the generators' noise
    (sigma = 0.1) and the PSNR definition must reproduce that."""
    fx = json.load(open(os.path.join(GOLDEN, "noisy_psnr.json")))
    clean, noisy = synth.polygon_image(256, 256, seed=11, noise=math.sqrt(fx["noise_variance"]))
    assert abs(synth.psnr(clean, noisy) - fx["paper_psnr_db"]) < fx["tolerance_db"]

"""Pins of the guided-filter oracle (Section 3: Algorithm 1 and the matrix of Eqs. 5-6)
against the formula as printed, brute force, closed forms and invariants -- never against
the CUDA path."""
import itertools

import numpy as np
import pytest

from oracle import guided


def _brute_box(v, shape, r):
    ny, nx = shape
    V = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    out = np.zeros_like(V)
    ry = r if ny > 1 else 0
    for y, x in itertools.product(range(ny), range(nx)):
        vals = [V[y + dy, x + dx] for dy in range(-ry, ry + 1) for dx in range(-r, r + 1)
                if 0 <= y + dy < ny and 0 <= x + dx < nx]
        out[y, x] = sum(vals) / len(vals)
    return out.reshape(-1)


CASES = [((1, 25), 2, 0.01), ((7, 9), 1, 0.05), ((8, 6), 2, 1e-3)]


@pytest.mark.parametrize("shape,r,eps", CASES)
def test_box_mean_brute_force(shape, r, eps):
    v = np.random.default_rng(1).standard_normal(shape[0] * shape[1])
    np.testing.assert_allclose(guided.box_mean(v, shape, r), _brute_box(v, shape, r), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("shape,r,eps", CASES)
def test_algorithm1_is_the_matrix_of_eq6(shape, r, eps):
    """Eq. 5: the output of Algorithm 1 is a fixed matrix applied to x (D^-1 Wt with the
    border reading), for any x."""
    rng = np.random.default_rng(2)
    n = shape[0] * shape[1]
    g = rng.uniform(0, 1, n)
    G = guided.GuidedGraph(g, shape, r, eps)
    for _ in range(3):
        x = rng.standard_normal(n)
        np.testing.assert_allclose(guided.guided_filter(x, g, shape, r, eps), G.DINV_W @ x,
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape,r,eps", CASES)
def test_graph_symmetric_degree_is_window_count_laplacian_psd(shape, r, eps):
    g = np.random.default_rng(3).uniform(0, 1, shape[0] * shape[1])
    G = guided.GuidedGraph(g, shape, r, eps)
    assert abs(G.W - G.W.T).max() < 1e-15
    np.testing.assert_allclose(G.d, G.N, rtol=1e-13)
    ndim = 1 if shape[0] == 1 else 2
    N = G.N.reshape(shape)
    assert N.max() == (2 * r + 1) ** ndim                   # interior windows are full
    assert N.reshape(-1)[0] == (r + 1) ** ndim                # corner
    Ld = G.L.toarray()
    assert np.abs(Ld @ np.ones(G.n)).max() < 1e-12
    assert np.linalg.eigvalsh(Ld).min() > -1e-12


def test_interior_entries_equal_eq6_as_printed():
    """Away from the border every window has |omega| pixels and Eq. 6 (1 / |omega|^2, sum
    over the windows containing both pixels) equals Wt / |omega|."""
    shape, r, eps = (11, 12), 1, 0.02
    ny, nx = shape
    rng = np.random.default_rng(4)
    g = rng.uniform(0, 1, ny * nx)
    G = guided.GuidedGraph(g, shape, r, eps)
    Wd = G.W.toarray()
    om = (2 * r + 1) ** 2
    Gi = g.reshape(ny, nx)
    for (yi, xi), (dy, dx) in [((5, 5), (0, 1)), ((5, 6), (1, -1)), ((4, 7), (2, 2)), ((6, 4), (0, 0))]:
        yj, xj = yi + dy, xi + dx
        tot = 0.0
        for ky in range(r, ny - r):
            for kx in range(r, nx - r):
                if max(abs(yi - ky), abs(xi - kx)) <= r and max(abs(yj - ky), abs(xj - kx)) <= r:
                    win = Gi[ky - r:ky + r + 1, kx - r:kx + r + 1]
                    mu, var = win.mean(), win.var()
                    tot += 1.0 + (Gi[yi, xi] - mu) * (Gi[yj, xj] - mu) / (var + eps)
        eq6 = tot / om ** 2
        assert abs(Wd[yi * nx + xi, yj * nx + xj] / om - eq6) < 1e-14


def test_large_eps_and_constant_guide_give_box_of_box():
    """eps -> inf (or a constant guide: var = cov = 0) gives a = 0, b = mean_x, so the filter
    is the mean filter applied twice."""
    shape, r = (9, 10), 1
    rng = np.random.default_rng(5)
    x = rng.standard_normal(90)
    bb = guided.box_mean(guided.box_mean(x, shape, r), shape, r)
    g = rng.uniform(0, 1, 90)
    np.testing.assert_allclose(guided.guided_filter(x, g, shape, r, 1e14), bb, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(guided.guided_filter(x, np.full(90, 0.3), shape, r, 1e-2), bb, rtol=1e-13, atol=1e-14)


def test_self_guided_small_eps_preserves_a_step_edge():
    """Self-guided with eps -> 0: a window across the edge has a = var / (var + eps) -> 1 and
    b -> 0, a flat window a = 0 and b = its value, so a piecewise-constant image is kept."""
    shape = (8, 10)
    x = np.zeros(shape)
    x[:, 5:] = 1.0
    x = x.reshape(-1)
    y = guided.guided_filter(x, x, shape, 2, 1e-10)
    np.testing.assert_allclose(y, x, atol=1e-8)


def test_cg_on_the_guided_graph_is_krylov_optimal():
    """Algorithm 2 on the guided filter's L (Section 3 feeds it to the same filters): with
    T = D^-1 the iterate minimises x^T L x over x0 + K_k(D^-1 L, D^-1 r0), by brute force."""
    from oracle import solvers
    shape, r, k = (6, 7), 1, 5
    rng = np.random.default_rng(6)
    g = rng.uniform(0, 1, 42)
    G = guided.GuidedGraph(g, shape, r, 0.02)
    x0 = g.copy()
    out = solvers.cg(G, x0, k)
    Lm = G.L.toarray()
    M = Lm / G.d[:, None]
    V = [-(Lm @ x0) / G.d]
    for _ in range(k - 1):
        V.append(M @ V[-1])
    V, _ = np.linalg.qr(np.array(V).T)
    c = np.linalg.lstsq(V.T @ Lm @ V, -(V.T @ Lm @ x0), rcond=None)[0]
    np.testing.assert_allclose(out["x"], x0 + V @ c, rtol=1e-9, atol=1e-10)


def test_lobpcg_on_the_guided_graph_reaches_the_dense_pencil():
    """Algorithm 3 for the pencil (L, D) of the guided graph converges to the smallest
    generalised eigenvalues of the dense pencil."""
    import scipy.linalg as sla

    from oracle import solvers
    shape, r = (7, 8), 1
    rng = np.random.default_rng(8)
    g = rng.uniform(0, 1, 56)
    G = guided.GuidedGraph(g, shape, r, 0.05)
    X0 = rng.standard_normal((56, 3))
    out = solvers.lobpcg(G, X0, 60, tol=1e-11)
    lam = sla.eigh(G.L.toarray(), np.diag(G.d), eigvals_only=True)[:3]
    np.testing.assert_allclose(out["theta"], lam, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("shape,r", [((1, 30), 3), ((9, 11), 2)])
def test_difference_form_equals_the_laplacian(shape, r):
    """The identity the operator kernels use: with d_k = sum_j (x_j - x_k) / N_k and
    a_k = sum_j (g_j - mu_k)(x_j - x_k) / N_k / (sigma_k^2 + eps) over window k,
    (L x)_i = sum over windows k containing i of (x_i - x_k) - d_k - (g_i - mu_k) a_k."""
    ny, nx = shape
    rng = np.random.default_rng(9)
    g = rng.uniform(0, 1, ny * nx)
    x = rng.standard_normal(ny * nx)
    eps = 0.03
    G = guided.GuidedGraph(g, shape, r, eps)
    ry = r if ny > 1 else 0
    Gi, Xi = g.reshape(ny, nx), x.reshape(ny, nx)
    dk = np.zeros((ny, nx))
    ak = np.zeros((ny, nx))
    mu = np.zeros((ny, nx))
    for ky, kx in itertools.product(range(ny), range(nx)):
        mem = [(ky + dy, kx + dx) for dy in range(-ry, ry + 1) for dx in range(-r, r + 1)
               if 0 <= ky + dy < ny and 0 <= kx + dx < nx]
        gv = np.array([Gi[p] for p in mem])
        xv = np.array([Xi[p] for p in mem])
        mu[ky, kx] = gv.mean()
        var = ((gv - gv.mean()) ** 2).mean()
        dk[ky, kx] = (xv - Xi[ky, kx]).mean()
        ak[ky, kx] = ((gv - gv.mean()) * (xv - Xi[ky, kx])).mean() / (var + eps)
    lx = np.zeros((ny, nx))
    for iy, ix in itertools.product(range(ny), range(nx)):
        for dy in range(-ry, ry + 1):
            for dx in range(-r, r + 1):
                ky, kx = iy + dy, ix + dx
                if 0 <= ky < ny and 0 <= kx < nx:
                    lx[iy, ix] += (Xi[iy, ix] - Xi[ky, kx]) - dk[ky, kx] - (Gi[iy, ix] - mu[ky, kx]) * ak[ky, kx]
    np.testing.assert_allclose(lx.reshape(-1), G.L @ x, rtol=1e-11, atol=1e-12)

"""Pins of the oracle's filters (Sections 4-6: simple iteration, Algorithm 2, Algorithm 3)
against closed forms, brute force, library routines and invariants -- never against the
CUDA path."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import solvers, spectral
from oracle.graph import Graph
from paper_1509_02468_gb300 import synth


def _graph_1d(n=60, seed=0, r=2, ss=1.5, sr=0.15):
    _, noisy = synth.signal_1d(n, seed, segments=4, min_len=8)
    return Graph(noisy, (1, n), r, ss, sr), noisy


def _graph_2d(ny=9, nx=10, seed=0, r=1, ss=1.0, sr=0.2):
    _, noisy = synth.polygon_image(ny, nx, seed, polygons=3, dtype=np.float64)
    return Graph(noisy, (ny, nx), r, ss, sr), noisy.reshape(-1)


# ------------------------------------------------------------------ simple iteration
def test_simple_iteration_is_spectral_power_filter():
    """Section 4: (D^-1 W)^k = (I - D^-1 L)^k, i.e. h(mu) = (1 - mu)^k in the graph Fourier
    basis of D^-1/2 L D^-1/2."""
    G, x0 = _graph_1d()
    xk = solvers.simple_iteration(G, x0, 7)
    ref, _ = spectral.spectral_filter(G, x0, lambda mu: (1.0 - mu) ** 7)
    np.testing.assert_allclose(xk, ref, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------ re-guided iteration
def _bf_step_brute(x, shape, r, ss, sr):
    """One step of Eq. 1 written out pixel by pixel: y_i = sum_j w_ij x_j / sum_j w_ij with
    w_ij of Eq. 2 over the in-image square window, guided by x itself."""
    ny, nx = shape
    X = np.asarray(x, dtype=np.float64).reshape(ny, nx)
    Y = np.zeros_like(X)
    ry = r if ny > 1 else 0
    for yi in range(ny):
        for xi in range(nx):
            num = den = 0.0
            for dy in range(-ry, ry + 1):
                for dx in range(-r, r + 1):
                    yj, xj = yi + dy, xi + dx
                    if 0 <= yj < ny and 0 <= xj < nx:
                        w = math.exp(-(dx * dx + dy * dy) / (2 * ss * ss)) * \
                            math.exp(-(X[yi, xi] - X[yj, xj]) ** 2 / (2 * sr * sr))
                        num += w * X[yj, xj]
                        den += w
            Y[yi, xi] = num / den
    return Y.reshape(-1)


@pytest.mark.parametrize("shape,r", [((1, 23), 2), ((7, 6), 1)])
def test_reguided_iteration_brute_force(shape, r):
    """Section 2, first way: every step re-guides by the previous result; three steps of the
    pixel-by-pixel Eq. 1 with the weights taken from the current iterate."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, 1.0, shape[0] * shape[1])
    ref = x.copy()
    for _ in range(3):
        ref = _bf_step_brute(ref, shape, r, 1.3, 0.25)
    got = solvers.reguided_iteration(x, shape, r, 1.3, 0.25, 3)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)


def test_reguided_iteration_without_range_term_is_linear():
    """With sigma_r = inf the weights of Eq. 2 do not depend on the guide, so re-guiding
    changes nothing: the cascade equals the fixed-weight iteration (Section 2, second way)."""
    G, x0 = _graph_2d(sr=np.inf)
    got = solvers.reguided_iteration(x0, G.shape, 1, 1.0, np.inf, 4)
    np.testing.assert_allclose(got, solvers.simple_iteration(G, x0, 4), rtol=1e-13, atol=1e-14)


def test_reguided_iteration_differs_from_fixed_weights_and_stays_in_range():
    """With a finite sigma_r the two ways of iterating differ (the nonlinear one re-weights),
    and every step is a convex combination: the iterates stay within [min x0, max x0]; a
    constant signal is a fixed point."""
    G, x0 = _graph_2d()
    nl = solvers.reguided_iteration(x0, G.shape, 1, 1.0, 0.2, 5)
    lin = solvers.simple_iteration(G, x0, 5)
    assert np.max(np.abs(nl - lin)) > 1e-6
    assert nl.min() >= x0.min() - 1e-15 and nl.max() <= x0.max() + 1e-15
    c = np.full(G.n, 0.37)
    np.testing.assert_allclose(solvers.reguided_iteration(c, G.shape, 1, 1.0, 0.2, 3), c, rtol=0, atol=1e-15)


def test_simple_iteration_keeps_d_weighted_mean():
    """e^T D (D^-1 W x) = d^T x: the BF step preserves the d-weighted sum."""
    G, x0 = _graph_2d()
    xk = solvers.simple_iteration(G, x0, 5)
    assert math.isclose(G.d @ xk, G.d @ x0, rel_tol=1e-13)


# ------------------------------------------------------------------ Algorithm 2
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_cg_is_krylov_optimal(k):
    """P6: with T = D^-1 and the flexible beta (s_old^T r_old), x_k minimises x^T L x over
    x0 + K_k(D^-1 L, D^-1 r0) -- brute force over the explicit Krylov basis."""
    G, x0 = _graph_1d(n=50, seed=3)
    out = solvers.cg(G, x0, k)
    assert out["iters"] == k
    Lm = G.dense("L")
    M = Lm / G.d[:, None]
    v = -(Lm @ x0) / G.d
    V = [v]
    for _ in range(k - 1):
        V.append(M @ V[-1])
    V = np.array(V).T
    V, _ = np.linalg.qr(V)
    c = np.linalg.lstsq(V.T @ Lm @ V, -(V.T @ Lm @ x0), rcond=None)[0]
    xref = x0 + V @ c
    np.testing.assert_allclose(out["x"], xref, rtol=1e-9, atol=1e-10)
    # and the energy is smaller than for the printed-beta variant or simple iteration
    e = lambda z: z @ Lm @ z
    assert e(out["x"]) <= e(solvers.simple_iteration(G, x0, k)) + 1e-14


def test_cg_matches_library_pcg_on_shifted_system():
    """Algorithm 2 applied to (L + s I) x = s x0 with T = D^-1 equals scipy's PCG after the
    same number of iterations (no early stop)."""
    G, x0 = _graph_2d(ny=8, nx=9, seed=2)
    s = 0.05
    k = 6
    out = solvers.cg(G, x0, k, shift=s)
    A = (G.L + s * __import__("scipy.sparse", fromlist=["identity"]).identity(G.n)).tocsr()
    Minv = spla.LinearOperator(A.shape, matvec=lambda v: v / G.d)
    xs, info = spla.cg(A, s * x0, x0=x0.copy(), rtol=1e-300, atol=0.0, maxiter=k, M=Minv)
    np.testing.assert_allclose(out["x"], xs, rtol=1e-10, atol=1e-12)


def test_cg_keeps_d_weighted_mean():
    """P7: r = -L x has e^T r = 0, so with T = D^-1 every p satisfies e^T D p = 0 and
    e^T D x_k = e^T D x0."""
    G, x0 = _graph_2d(seed=4)
    out = solvers.cg(G, x0, 12)
    assert math.isclose(G.d @ out["x"], G.d @ x0, rel_tol=1e-12)


@pytest.mark.parametrize("beta", ["sr", "ss"])
def test_cg_is_polynomial_filter(beta):
    """P8 (Section 5): x_k = chi_k(D^-1 L) x0, with chi_k built from CG's own alpha/beta by
    the scalar recurrences, evaluated through the eigendecomposition (Eq. 8)."""
    G, x0 = _graph_1d(n=70, seed=5)
    out = solvers.cg(G, x0, 9, beta=beta)
    ref, _ = spectral.spectral_filter(
        G, x0, lambda mu: spectral.cg_polynomial(out["alpha"], out["beta"], mu))
    np.testing.assert_allclose(out["x"], ref, rtol=1e-9, atol=1e-10)


def test_cg_printed_beta_equals_flexible_when_T_is_identity():
    """Section 5 reading: s_old^T s_old = s_old^T r_old when s = r (T = I)."""
    G, x0 = _graph_1d(n=40, seed=6)
    a = solvers.cg(G, x0, 8, precond="identity", beta="sr")
    b = solvers.cg(G, x0, 8, precond="identity", beta="ss")
    np.testing.assert_allclose(a["x"], b["x"], rtol=1e-13, atol=1e-14)


def test_cg_null_start_exits_at_once():
    """x0 in the null space of L: r = -L x0 = 0, so s^T r = 0 at once and x is returned
    unchanged (x0 = 0 exactly; a constant x0 up to the rounding of L e)."""
    G, _ = _graph_1d(n=30)
    out = solvers.cg(G, np.zeros(G.n), 5)
    assert out["iters"] == 0 and out["status"] == "converged"
    np.testing.assert_array_equal(out["x"], 0.0)
    out = solvers.cg(G, np.full(G.n, 0.3), 5)
    np.testing.assert_allclose(out["x"], 0.3, rtol=0, atol=1e-14)


def test_cg_tolerance_stops_on_shifted_system():
    G, x0 = _graph_2d(ny=10, nx=10, seed=8)
    out = solvers.cg(G, x0, 500, shift=0.1, tol=1e-10)
    assert out["status"] == "converged" and out["iters"] < 500
    A = G.dense("L") + 0.1 * np.eye(G.n)
    np.testing.assert_allclose(out["x"], np.linalg.solve(A, 0.1 * x0), rtol=1e-8, atol=1e-9)


# ------------------------------------------------------------------ Rayleigh-Ritz helper
def test_rayleigh_ritz_matches_library_generalised_eigensolver():
    rng = np.random.default_rng(0)
    m = 12
    Q = rng.standard_normal((m, m))
    GB = Q @ Q.T + m * np.eye(m)
    H = rng.standard_normal((m, m))
    GA = H + H.T
    theta, C, _ = solvers.rayleigh_ritz(GA, GB, 4)
    ref = sla.eigh(GA, GB, eigvals_only=True)[:4]
    np.testing.assert_allclose(theta, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(C.T @ GB @ C, np.eye(4), atol=1e-12)
    np.testing.assert_allclose(C.T @ GA @ C, np.diag(theta), atol=1e-11)


def test_rayleigh_ritz_rejects_dependent_basis():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((30, 4))
    S = np.hstack([S, S[:, :1] * 2.0])
    with pytest.raises(np.linalg.LinAlgError):
        solvers.rayleigh_ritz(S.T @ S, S.T @ S, 2)


# ------------------------------------------------------------------ Algorithm 3
def test_lobpcg_first_step_single_vector_closed_form():
    """P10: one LOBPCG step with k = 1 is Rayleigh-Ritz on span{x, w}, w = D^-1 (L x -
    lambda D x): the smaller root of the 2x2 pencil's quadratic det(GA - t GB) = 0."""
    G, x0 = _graph_1d(n=45, seed=9)
    out = solvers.lobpcg(G, x0.reshape(-1, 1), 1)
    L = G.dense("L")
    x = x0 / math.sqrt(x0 @ (G.d * x0))
    lam0 = x @ L @ x
    w = (L @ x - lam0 * G.d * x) / G.d
    S = np.stack([x, w], 1)
    A = S.T @ L @ S
    B = S.T @ (G.d[:, None] * S)
    qa = B[0, 0] * B[1, 1] - B[0, 1] ** 2
    qb = -(A[0, 0] * B[1, 1] + A[1, 1] * B[0, 0] - 2 * A[0, 1] * B[0, 1])
    qc = A[0, 0] * A[1, 1] - A[0, 1] ** 2
    t = (-qb - math.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    assert math.isclose(out["theta"][0], t, rel_tol=1e-10)
    assert math.isclose(out["theta_hist"][0][0], lam0, rel_tol=1e-12)


@pytest.mark.parametrize("pencil", ["D", "I"])
def test_lobpcg_converges_to_dense_eigenvalues(pencil):
    """P9: converged Ritz values equal the dense generalised eigenvalues; X^T B X = I,
    X^T L X = diag(theta); Ritz values never increase and never go below the exact ones."""
    G, x0 = _graph_2d(ny=10, nx=12, seed=10)
    k = 4
    X0 = synth.block_start(x0, k, seed=10)
    out = solvers.lobpcg(G, X0, 120, pencil=pencil)
    lam, _ = spectral.pencil_eig(G, pencil)
    np.testing.assert_allclose(out["theta"], lam[:k], rtol=1e-10, atol=1e-12)
    b = G.d if pencil == "D" else np.ones(G.n)
    X = out["X"]
    np.testing.assert_allclose(X.T @ (b[:, None] * X), np.eye(k), atol=1e-10)
    np.testing.assert_allclose(X.T @ G.L @ X, np.diag(out["theta"]), atol=1e-10)
    h = out["theta_hist"]
    assert np.all(np.diff(h, axis=0) <= 1e-12)
    assert np.all(h >= lam[None, :k] - 1e-12)
    assert out["resid"].max() < 1e-6


def test_lobpcg_constraint_gives_fiedler_value():
    """P9 with the e-constraint (Section 6): the smallest constrained Ritz value converges
    to lambda_2 of the pencil, and every iterate stays B-orthogonal to e."""
    G, x0 = _graph_1d(n=80, seed=11)
    X0 = synth.block_start(x0, 2, seed=11)
    out = solvers.lobpcg(G, X0, 150, constrain=True)
    lam, _ = spectral.pencil_eig(G, "D")
    np.testing.assert_allclose(out["theta"], lam[1:3], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(G.d @ out["X"], 0.0, atol=1e-10)


def test_lobpcg_path_graph_closed_form_B_identity():
    """P5 + P9: B = I, T = I on the path graph converges to 2 - 2 cos(pi j / n)."""
    n = 60
    G = Graph(np.zeros(n), (1, n), 1, np.inf, np.inf)
    X0 = synth.block_start(np.random.default_rng(3).standard_normal(n), 3, seed=3)
    out = solvers.lobpcg(G, X0, 300, pencil="I", precond="identity")
    ref = 2.0 - 2.0 * np.cos(np.pi * np.arange(3) / n)
    np.testing.assert_allclose(out["theta"], ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("constrain", [False, True])
def test_lobpcg_output_is_ideal_lowpass_when_converged(constrain):
    """A6 reading + Eq. 8: once converged, y is the exact spectral low-pass filter of x0
    (projection on the k lowest eigenvectors; with the constraint e plus the k lowest
    non-constant ones)."""
    G, x0 = _graph_2d(ny=9, nx=9, seed=12)
    k = 3
    X0 = synth.block_start(x0, k, seed=12)
    out = solvers.lobpcg(G, X0, 200, constrain=constrain)
    ref, lam = spectral.lowpass_projection(G, x0, k + (1 if constrain else 0))
    np.testing.assert_allclose(out["y"], ref, rtol=1e-7, atol=1e-8)


def test_lobpcg_tolerance_stops_early():
    G, x0 = _graph_1d(n=50, seed=13)
    out = solvers.lobpcg(G, synth.block_start(x0, 2, seed=13), 500, tol=1e-8)
    assert out["status"] == "converged" and out["iters"] < 500
    assert out["resid"].max() <= 1e-8


def test_filters_denoise_polygon_image():
    """P12 (Section 7, quality sanity, not parity): CG and LOBPCG filters raise the PSNR."""
    clean, noisy = synth.polygon_image(48, 48, seed=21, polygons=6, noise=0.1,
                                       dtype=np.float64)
    G = Graph(noisy, noisy.shape, 1, 1.0, 0.1, window="cross")
    x0 = noisy.reshape(-1)
    p0 = synth.psnr(clean.reshape(-1), x0)
    xcg = solvers.cg(G, x0, 20)["x"]
    assert synth.psnr(clean.reshape(-1), xcg) > p0 + 0.5


def test_lobpcg_orthogonal_p_spans_the_same_subspaces():
    """span{X_t+1, P_t+1} = span{X_t+1, X_t}: keeping P B-orthogonal to X changes no Ritz
    pair (raw P = [W P] C_WP as in Algorithm 3 gives the same trajectory)."""
    G, x0 = _graph_2d(ny=14, nx=15, seed=16)
    X0 = synth.block_start(x0, 3, seed=16)
    a = solvers.lobpcg(G, X0, 25, p_ortho=True)
    b = solvers.lobpcg(G, X0, 25, p_ortho=False)
    np.testing.assert_allclose(a["theta_hist"], b["theta_hist"], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(a["y"], b["y"], rtol=1e-8, atol=1e-10)

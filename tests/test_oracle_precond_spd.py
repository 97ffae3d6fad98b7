"""Pins of the oracle's symmetric positive definite preconditioner (oracle/precond_spd.py):
the correlation against an independent library routine, the adjoint identity, symmetry and
positive definiteness of T, the Jacobi special case, the loss gradient against central
finite differences, and CG with this T minimising the A-norm of the error over its Krylov
space (the optimality Section 5 relies on), by brute force."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy import signal

from oracle import precond_spd as ps
from oracle import solvers
from oracle.graph import Graph


def _image(ny=9, nx=11, seed=0):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0, 1, (ny, nx))
    return g


@pytest.mark.parametrize("half", [1, 2, 3])
def test_correlate_is_zero_padded_cross_correlation(half):
    rng = np.random.default_rng(half)
    x = rng.standard_normal((8, 13))
    K = rng.standard_normal((2 * half + 1, 2 * half + 1))
    ref = signal.correlate2d(x, K, mode="same", boundary="fill")
    np.testing.assert_allclose(ps.correlate(x, K), ref, atol=1e-12)


def test_correlate_adjoint_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((10, 7))
    y = rng.standard_normal((10, 7))
    K = rng.standard_normal((7, 7))                      # wider than the image is tall
    lhs = np.sum(ps.correlate(x, K) * y)
    rhs = np.sum(x * ps.correlate_adjoint(y, K))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_T_is_symmetric_positive_definite_and_jacobi_at_zero():
    g = _image()
    G = Graph(g, g.shape, 2, 2.0, 0.1)
    rng = np.random.default_rng(4)
    K = 0.3 * rng.standard_normal((5, 5))
    T = ps.matrix(K, G.d, g.shape)
    np.testing.assert_allclose(T, T.T, atol=1e-13)
    lam = np.linalg.eigvalsh(0.5 * (T + T.T))
    assert lam.min() >= (1.0 / G.d.max()) * (1 - 1e-12)  # I + K^T K >= I
    # K = 0: Jacobi; K = c * delta: (1 + c^2) D^-1
    r = rng.standard_normal(G.n)
    np.testing.assert_allclose(ps.apply(ps.identity_kernel(2), G.d, g.shape, r), r / G.d, rtol=1e-14)
    np.testing.assert_allclose(ps.apply(ps.identity_kernel(3, 0.5), G.d, g.shape, r), 1.25 * r / G.d, rtol=1e-14)
    # a block is mapped column by column
    R = rng.standard_normal((G.n, 3))
    Y = ps.apply(K, G.d, g.shape, R)
    np.testing.assert_allclose(Y[:, 1], T @ R[:, 1], atol=1e-13)


@pytest.mark.parametrize("half", [1, 3])
def test_loss_gradient_matches_central_differences(half):
    g = _image(8, 10, seed=5)
    G = Graph(g, g.shape, 2, 2.0, 0.1)
    sigma = 0.05
    A = (G.L + sigma * sp.identity(G.n)).tocsr()
    rng = np.random.default_rng(6)
    r = rng.standard_normal(G.n)
    z = np.linalg.solve(A.toarray(), r)
    K = 0.2 * rng.standard_normal((2 * half + 1, 2 * half + 1))
    loss, grad = ps.loss_grad(K, G.d, g.shape, A, r, z)
    # the loss is the A-norm of the error, relative
    e = z - ps.apply(K, G.d, g.shape, r)
    assert loss == pytest.approx(float(e @ (A @ e)) / float(z @ (A @ z)), rel=1e-13)
    eps = 1e-6
    fd = np.zeros_like(K)
    for a in range(K.shape[0]):
        for b in range(K.shape[1]):
            Kp, Km = K.copy(), K.copy()
            Kp[a, b] += eps
            Km[a, b] -= eps
            fd[a, b] = (ps.loss_grad(Kp, G.d, g.shape, A, r, z)[0] - ps.loss_grad(Km, G.d, g.shape, A, r, z)[0]) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-9 * np.abs(fd).max())


def test_cg_with_spd_T_minimises_the_energy_error_over_its_krylov_space():
    """x_k of Algorithm 2 with this T on A x = b (A = L + sigma I, b = sigma x0) is the
    minimiser of ||x - x*||_A over x0 + span{T r0, (T A) T r0, ...} (brute force)."""
    g = _image(7, 8, seed=7)
    G = Graph(g, g.shape, 1, 2.0, 0.2)
    sigma = 0.1
    A = (G.L + sigma * sp.identity(G.n)).toarray()
    x0 = g.reshape(-1)
    b = sigma * x0
    xs = np.linalg.solve(A, b)
    rng = np.random.default_rng(8)
    K = 0.4 * rng.standard_normal((3, 3))
    T = lambda v: ps.apply(K, G.d, g.shape, v)
    r0 = b - A @ x0
    for k in (1, 3, 6):
        out = solvers.cg(G, x0, k, precond=T, shift=sigma)
        V = [T(r0)]
        for _ in range(k - 1):
            V.append(T(A @ V[-1]))
        V = np.linalg.qr(np.stack(V, axis=1))[0]
        c = np.linalg.solve(V.T @ A @ V, V.T @ A @ (xs - x0))
        x_opt = x0 + V @ c
        np.testing.assert_allclose(out["x"], x_opt, atol=1e-9 * np.abs(x_opt).max())

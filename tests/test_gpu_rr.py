"""The FP64 Rayleigh-Ritz step of LOBPCG on the GPU (Algorithm 3's "Rayleigh-Ritz method
for the pencil on the trial subspace") against the oracle's Rayleigh-Ritz, on random
pencils of every size the LOBPCG driver uses, clustered spectra, and dependent bases."""
import numpy as np
import pytest
import torch

from oracle import solvers
from tests.gpu_helpers import bf, host

pytestmark = pytest.mark.gpu


def pencil(m, seed, cluster=False, scale_range=3.0, lam=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    lam_b = 10 ** rng.uniform(-1, 1, m)
    GB = (Q * lam_b) @ Q.T
    s = 10 ** rng.uniform(-scale_range, scale_range, m)       # badly scaled basis vectors
    GB = GB * s[:, None] * s[None, :]
    Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
    if lam is None:
        lam = np.sort(np.concatenate([10 ** rng.uniform(-6, -2, m // 3 + 1), rng.uniform(0.1, 2.0, m)]))[:m]
    if cluster and m >= 6:
        lam[1] = lam[0] * (1 + 1e-9)
        lam[3] = lam[2] * (1 + 1e-7)
    # G_A = G_B^{1/2} Q2 diag(lam) Q2^T G_B^{1/2}: the pencil's eigenvalues are lam
    w, V = np.linalg.eigh(GB)
    Bh = (V * np.sqrt(w)) @ V.T
    GA = Bh @ (Q2 * lam) @ Q2.T @ Bh
    return 0.5 * (GA + GA.T), 0.5 * (GB + GB.T), lam


def check(GA, GB, k, C, theta, tol=1e-9):
    C = host(C)
    th = host(theta)
    ref, Cref, _ = solvers.rayleigh_ritz(GA, GB, k)
    scale = np.maximum(np.abs(ref), 1e-12 * np.abs(ref).max() + 1e-300)
    assert np.max(np.abs(th - ref) / scale) < tol, (th, ref)
    np.testing.assert_allclose(C.T @ GB @ C, np.eye(k), atol=1e-9)
    np.testing.assert_allclose(C.T @ GA @ C, np.diag(th), atol=1e-9 * max(1.0, np.abs(th).max()))


@pytest.mark.parametrize("m,k", [(1, 1), (2, 1), (3, 1), (4, 2), (12, 4), (24, 8), (48, 16),
                                 (64, 32), (93, 31), (96, 32)])
@pytest.mark.parametrize("cluster", [False, True])
def test_rayleigh_ritz_matches_oracle(m, k, cluster):
    GA, GB, lam = pencil(m, seed=m * 7 + k, cluster=cluster)
    C, theta, _, status, restarts = bf().rayleigh_ritz(torch.as_tensor(GA).cuda(),
                                                       torch.as_tensor(GB).cuda(), k)
    assert status == 0 and restarts == 0
    check(GA, GB, k, C, theta)


def test_rayleigh_ritz_drops_dependent_p_block():
    k = 4
    rng = np.random.default_rng(3)
    S = rng.standard_normal((200, 2 * k))
    S = np.hstack([S, S[:, :k] @ rng.standard_normal((k, k))])   # P inside span X
    A = np.diag(rng.uniform(0.1, 1, 200))
    GA, GB = S.T @ A @ S, S.T @ S
    C, theta, _, status, restarts = bf().rayleigh_ritz(torch.as_tensor(GA).cuda(),
                                                       torch.as_tensor(GB).cuda(), k, m_nop=2 * k)
    assert status == 0 and restarts == 1
    assert np.all(host(C)[2 * k:] == 0)
    check(GA[:2 * k, :2 * k], GB[:2 * k, :2 * k], k, C[:2 * k], theta)


def test_rayleigh_ritz_reports_breakdown():
    k = 2
    rng = np.random.default_rng(4)
    S = rng.standard_normal((50, 3))
    S = np.hstack([S, S[:, :1]])
    GA, GB = S.T @ S, S.T @ S
    _, _, _, status, _ = bf().rayleigh_ritz(torch.as_tensor(GA).cuda(), torch.as_tensor(GB).cuda(), k)
    assert status == 2


def test_next_p_is_b_orthogonal_to_ritz_vectors():
    k = 8
    GA, GB, _ = pencil(3 * k, seed=11)
    C, theta, Cp, status, _ = bf().rayleigh_ritz(torch.as_tensor(GA).cuda(), torch.as_tensor(GB).cuda(),
                                                 k, want_cp=True)
    C, Cp = host(C), host(Cp)
    np.testing.assert_allclose(C.T @ GB @ Cp, 0.0, atol=1e-10)
    # Cp spans the same directions as the W/P part of C, up to X
    Cw = C.copy()
    Cw[:k] = 0
    Z = C.T @ GB @ Cw
    np.testing.assert_allclose(Cp, Cw - C @ Z, atol=1e-10)


@pytest.mark.parametrize("m,k,gap", [(48, 16, 2e-6), (24, 8, 1e-6), (96, 30, 1e-6)])
def test_rayleigh_ritz_cluster_across_the_kth_eigenvalue(m, k, gap):
    """Eigenvalues k and k + 1 (and k + 2) of the pencil closer together than the
    neighbourhood the FP64 correction leaves alone (64 eps_32 |M|, about 1e-5 here): the k
    wanted Ritz vectors must span the oracle's invariant subspace (the B-orthogonal
    projectors agree), not a mixture with the unwanted neighbours.  Gaps of a few eps_32 |M|
    (3e-7 here) are below this bar: their FP32 inverse-iteration vectors can lose a
    direction of the cluster (measured projector error 1e-5)."""
    rng = np.random.default_rng(m + k)
    lam = np.sort(rng.uniform(0.05, 1.9, m))
    lam[k] = lam[k - 1] + gap
    lam[k + 1] = lam[k] + gap
    lam = np.sort(lam)
    GA, GB, _ = pencil(m, seed=5 * m + k, scale_range=1.0, lam=lam)
    C, theta, _, status, _ = bf().rayleigh_ritz(torch.as_tensor(GA).cuda(), torch.as_tensor(GB).cuda(), k)
    assert status == 0
    check(GA, GB, k, C, theta)
    _, Cref, _ = solvers.rayleigh_ritz(GA, GB, k)
    P, Pref = host(C) @ host(C).T @ GB, Cref @ Cref.T @ GB
    assert np.linalg.norm(P - Pref) <= 1e-6 * np.sqrt(k), np.linalg.norm(P - Pref)

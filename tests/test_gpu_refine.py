"""The shifted system (L + sigma I) x = sigma x0 (the Tikhonov form of the CG filter,
Algorithm 2 with a shift) on the GPU: the residual entry point against the FP64 oracle,
and the mixed-precision refinement checked by the oracle's own FP64 matrices."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from tests.gpu_helpers import TOL_F32, TOL_F64, bf, dev, host, image_case, make_pair, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_shifted_residual_matches_oracle(dtype):
    _, g = image_case(57, 83, 51, dtype=np.float64 if dtype == torch.float64 else np.float32)
    G, O = make_pair(g, 3, 2.0, 0.08, dtype=dtype)
    rng = np.random.default_rng(4)
    x0 = g.reshape(-1).astype(np.float64)
    x = x0 + 0.01 * rng.standard_normal(x0.size)
    x0d, xd = dev(x0, dtype), dev(x, dtype)
    sigma = 1e-2
    r = host(bf().shifted_residual(G, x0d, xd, sigma))
    ref = sigma * (host(x0d) - host(xd)) - O.L @ host(xd)
    assert rel_l2(r, ref) <= (TOL_F64 if dtype == torch.float64 else TOL_F32)


def _true_rel_residual(O, x0, x, sigma):
    A = (O.L + sigma * sp.identity(O.n, format="csr")).tocsr()
    b = sigma * x0
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


@pytest.mark.parametrize("precond", ["jacobi", "identity"])
def test_refinement_reaches_true_residual(precond):
    _, g = image_case(160, 160, 52)
    G32, O = make_pair(g, 3, 2.0, 0.08)
    G64 = bf().bf_weights(dev(g, torch.float64), 3, 2.0, 0.08)
    x0 = g.reshape(-1).astype(np.float64)
    sigma, tol = 1e-2, 1e-7
    x, info = bf().cg_refine(G64, G32, dev(x0, torch.float64), sigma, tol, precond=precond)
    assert info.status == "converged"
    rel = _true_rel_residual(O, x0, host(x), sigma)
    assert rel <= tol * 1.01
    assert abs(info.rnorm / info.ref - rel) <= 1e-2 * rel + 1e-12
    # the solution itself, against a direct FP64 solve of the oracle's system
    A = (O.L + sigma * sp.identity(O.n, format="csr")).tocsc()
    exact = spla.spsolve(A, sigma * x0)
    assert rel_l2(host(x), exact) <= 1e-5

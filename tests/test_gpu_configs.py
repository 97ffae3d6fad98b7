"""Parity at the sizes of the batched and the shifted-system workloads.

* The 256-instance batch (192 images with sides log-uniform in [64, 1024], 64 signals with
  lengths log-uniform in [1e3, 1e6], 36.7 M samples): one bf_batch_cg run of 50 Jacobi CG
  iterations (Algorithm 2), every instance compared in full with the FP64 oracle's CG
  (the oracle runs in a pool of spawned worker processes).
* The 1024 x 1024 image of the shifted-system workload: cg_filter on (L + sigma I) x =
  sigma x0 with sigma = 1e-2, at a fixed iteration count and with the tolerance the
  refinement's inner solves use, against the oracle; and cg_refine to a true residual of
  1e-5, checked with the oracle's FP64 matrices.
"""
import numpy as np
import pytest
import torch

from paper_1509_02468_gb300 import synth
from tests.gpu_helpers import TOL_F32, bf, dev, host, rel_l2

pytestmark = pytest.mark.gpu

from tests.oracle_jobs import (BATCH_SEED, CG_ITERS, batch_cg_error, batch_instance, batch_lobpcg_error,
                               oracle_pool)


def test_batch_256_instances_every_instance_against_oracle():
    sizes = synth.batch_sizes(BATCH_SEED)
    assert len(sizes) == 256
    graphs, x0s = [], []
    for i, (nd, ny, nx) in enumerate(sizes):
        noisy, (r, ss, sr) = batch_instance(i, nd, ny, nx)
        t = dev(noisy)
        graphs.append(bf().bf_weights(t, r, ss, sr))
        x0s.append(t.reshape(-1))
    B = bf().Batch(graphs)
    outs, infos = B.cg(x0s, CG_ITERS)
    # the persistent (one cooperative launch) form gives the same results exactly
    outs_p, infos_p = B.cg_persistent(x0s, CG_ITERS)
    assert all(torch.equal(a, b) for a, b in zip(outs, outs_p))
    assert all(a.iters == b.iters for a, b in zip(infos, infos_p))
    jobs = [(i, nd, ny, nx, host(x)) for i, ((nd, ny, nx), x) in enumerate(zip(sizes, outs))]
    for G in graphs:
        G.free()
    with oracle_pool() as ex:
        # largest instances first, so the pool finishes evenly
        order = sorted(jobs, key=lambda j: -j[2] * j[3])
        results = list(ex.map(batch_cg_error, order, chunksize=1))
    worst = max(results, key=lambda t: t[2])
    for i, iters, err in results:
        assert infos[i].iters == iters == CG_ITERS
        assert err <= TOL_F32, (i, sizes[i], err)
    assert worst[2] <= TOL_F32


def test_shifted_cg_1024_fixed_count_and_inner_tolerance():
    from oracle import solvers
    from oracle.graph import Graph
    _, noisy = synth.polygon_image(1024, 1024, 5)
    t = dev(noisy)
    G = bf().bf_weights(t, 3, 2.0, 0.08)
    O = Graph(noisy.astype(np.float64), noisy.shape, 3, 2.0, 0.08)
    x0 = noisy.reshape(-1).astype(np.float64)
    sigma = 1e-2
    # a fixed count
    x, info, _ = bf().cg_filter(G, t.reshape(-1), 100, shift=sigma)
    ref = solvers.cg(O, x0, 100, shift=sigma)
    assert info.iters == ref["iters"] == 100
    assert rel_l2(host(x), ref["x"]) <= TOL_F32
    # with the inner tolerance of the mixed-precision refinement: the GPU's FP32 recursive
    # residual and the oracle's FP64 one cross 1e-3 at the same iteration (+-1); the GPU
    # iterate equals the oracle's after as many iterations
    x, info, _ = bf().cg_filter(G, t.reshape(-1), 1000, shift=sigma, tol=1e-3)
    ref = solvers.cg(O, x0, 1000, shift=sigma, tol=1e-3)
    assert info.status == ref["status"] == "converged"
    assert abs(info.iters - ref["iters"]) <= 1
    same = solvers.cg(O, x0, info.iters, shift=sigma)
    assert rel_l2(host(x), same["x"]) <= TOL_F32
    # the same system to a TRUE relative residual of 1e-5 by mixed-precision refinement
    # (FP64 residuals, FP32 inner CG to 1e-3), checked with the oracle's FP64 matrices
    import scipy.sparse as sp
    G64 = bf().bf_weights(dev(noisy, torch.float64), 3, 2.0, 0.08)
    x, info = bf().cg_refine(G64, G, dev(x0, torch.float64), sigma, 1e-5)
    assert info.status == "converged"
    A = (O.L + sigma * sp.identity(O.n, format="csr")).tocsr()
    rel = float(np.linalg.norm(sigma * x0 - A @ host(x)) / np.linalg.norm(sigma * x0))
    assert rel <= 1.01e-5



def test_batch_256_instances_lobpcg():
    """Block LOBPCG (k = 16, 30 iterations) on all 256 instances over a pool of streams:
    every instance equals its own lobpcg_filter call exactly; the instances of at most
    2^16 samples are compared with the oracle: the filtered signal to the FP32 bar 1e-5,
    the Ritz values by the A8 reading (1e-6) or, for the tiny smallest Ritz values of small
    instances (A8 floor below 1e-5), to 1e-6 of the pencil's norm (TOL_RITZ_ABS: the FP32
    Gram entries carry absolute errors of order 2^-24 times the pencil's spectral radius,
    < 2, and Weyl's inequality bounds the Ritz values' absolute error by the norm of the
    m x m error matrix)."""
    from tests.gpu_helpers import TOL_F32, TOL_RITZ, TOL_RITZ_ABS
    sizes = synth.batch_sizes(BATCH_SEED)
    graphs, X0s = [], []
    for i, (nd, ny, nx) in enumerate(sizes):
        noisy, (r, ss, sr) = batch_instance(i, nd, ny, nx)
        t = dev(noisy)
        graphs.append(bf().bf_weights(t, r, ss, sr))
        X0s.append(dev(synth.block_start(noisy.reshape(-1), 16, seed=4000 + i)))
    B = bf().Batch(graphs)
    thetas, ys, infos = B.lobpcg(X0s, 30, nstreams=32)
    for G, X0, th, y, info in zip(graphs, X0s, thetas, ys, infos):
        single = bf().lobpcg_filter(G, X0, 30, want_X=False)
        assert torch.equal(th, single["theta"]) and torch.equal(y, single["y"])
        assert info.iters == 30
    jobs = [(i, nd, ny, nx, host(X0s[i]), 30, host(thetas[i]), host(ys[i]))
            for i, (nd, ny, nx) in enumerate(sizes) if ny * nx <= 1 << 16]
    with oracle_pool() as ex:
        results = list(ex.map(batch_lobpcg_error, sorted(jobs, key=lambda j: -j[2] * j[3]), chunksize=1))
    assert len(results) >= 100
    worst_abs = max(r[3] for r in results if r[1] > TOL_RITZ) if any(r[1] > TOL_RITZ for r in results) else 0.0
    print(f"largest absolute Ritz-value error below the A8 floor: {worst_abs:.2e}")
    for i, e_th, e_y, e_abs, _ in results:
        assert e_th <= TOL_RITZ or e_abs <= TOL_RITZ_ABS, (i, sizes[i], e_th, e_abs)
        assert e_y <= TOL_F32, (i, sizes[i], e_y)

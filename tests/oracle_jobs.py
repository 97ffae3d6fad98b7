"""Oracle work for the configuration-size GPU tests, run in spawned worker processes
(imports numpy and the oracle only: no torch, no CUDA)."""
import numpy as np

from paper_1509_02468_gb300 import synth

BATCH_SEED, CG_ITERS = 4, 50


def batch_instance(i, nd, ny, nx):
    """The mixed batch's instance i as the benchmark generates it (seed 4000 + i), with its
    window radius, sigma_s and sigma_r."""
    if nd == 2:
        _, noisy = synth.polygon_image(ny, nx, 4000 + i, noise=0.05)
        return noisy, (3, 2.0, 0.08)
    _, noisy = synth.signal_1d(nx, 4000 + i, noise=0.1, dtype=np.float32)
    return noisy, (5, 3.0, 0.1)


def batch_cg_error(job):
    """(i, oracle iterations, relative L2 error of x_gpu) for the oracle's CG on instance i."""
    from oracle import solvers
    from oracle.graph import Graph
    i, nd, ny, nx, x_gpu = job
    noisy, (r, ss, sr) = batch_instance(i, nd, ny, nx)
    g64 = np.asarray(noisy, np.float32).astype(np.float64)
    ref = solvers.cg(Graph(g64, (ny, nx), r, ss, sr), g64.reshape(-1), CG_ITERS)
    x = np.asarray(x_gpu, np.float64).reshape(-1)
    return i, ref["iters"], float(np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]))


def batch_lobpcg_error(job):
    """(i, Ritz-value error by the A8 reading, relative L2 error of y, largest absolute
    Ritz-value error, the oracle's Ritz value where the A8 error is largest) of the GPU
    results against the oracle's LOBPCG(k, kmax) on instance i from the given FP32 block
    start."""
    from oracle import solvers
    from oracle.graph import Graph
    i, nd, ny, nx, X0, kmax, theta, y = job
    noisy, (r, ss, sr) = batch_instance(i, nd, ny, nx)
    g64 = np.asarray(noisy, np.float32).astype(np.float64)
    ref = solvers.lobpcg(Graph(g64, (ny, nx), r, ss, sr), np.asarray(X0, np.float64), kmax)
    th_ref = ref["theta"]
    scale = np.maximum(np.abs(th_ref), 1e-3 * np.abs(th_ref).max())
    dth = np.abs(np.asarray(theta, np.float64) - th_ref)
    e_th = float(np.max(dth / scale))
    e_y = float(np.linalg.norm(np.asarray(y, np.float64) - ref["y"]) / np.linalg.norm(ref["y"]))
    return i, e_th, e_y, float(dth.max()), float(th_ref[int(np.argmax(dth / scale))])

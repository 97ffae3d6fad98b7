"""Oracle work for the configuration-size GPU tests, run in spawned worker processes
(imports numpy and the oracle only: no torch, no CUDA)."""
import contextlib
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from paper_1509_02468_gb300 import synth

BATCH_SEED, CG_ITERS = 4, 50
_ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


@contextlib.contextmanager
def oracle_pool():
    """A pool of spawned workers (one per host core but one), each with one BLAS thread:
    the workers inherit the environment when they start, and without the limit every
    worker's BLAS would start a thread per core."""
    saved = {v: os.environ.get(v) for v in _ONE_THREAD}
    os.environ.update({v: "1" for v in _ONE_THREAD})
    try:
        workers = max(1, min(16, (os.cpu_count() or 2) - 1))
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            yield ex
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


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

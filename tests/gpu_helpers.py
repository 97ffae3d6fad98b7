"""Shared helpers for the GPU parity tests (CUDA path through the C-ABI vs the FP64 oracle)."""
import numpy as np
import torch

from oracle.graph import Graph
from paper_1509_02468_gb300 import synth

# Tolerances: relative L2 error of FP32 filter outputs (<= 1e-5) and of Ritz values
# (<= 1e-6, with the floor 1e-3 * theta_max for eigenvalues near 0); FP64 paths are held
# to rounding level.
TOL_F32 = 1e-5
TOL_F64 = 1e-11
TOL_RITZ = 1e-6
# Short, unconverged FP32 LOBPCG runs on small problems: FP32 vectors move the trajectory
# itself.  Emulating FP32 storage of X, W, P, AX, AW, AP inside the FP64 oracle moves the
# Ritz values of these cases by up to 4.6e-7 per step; the operator's FP32 window sums,
# followed by the cancellation in R = AX - B X theta, add a few times that on the GPU
# (up to 1.7e-6 measured).  The configuration-size runs are held to TOL_RITZ.
TOL_RITZ_SMALL_F32 = 3e-6
# Ritz values below the A8 floor (the tiny smallest eigenvalues of small instances, where
# 1e-3 theta_max is below 1e-5): 1e-6 relative to the norm of the pencil (L, D), whose
# spectral radius is below 2 (Gershgorin on D^-1 L).  The FP32 Gram products carry absolute
# errors of order 2^-24 times that radius per entry, and Weyl's inequality passes the norm
# of the m x m error matrix (up to m times an entry) to the Ritz values, so there the
# reachable accuracy is absolute, not relative to theta.
TOL_RITZ_ABS = 2e-6


def bf():
    from paper_1509_02468_gb300 import bf as _bf
    return _bf


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def tol_for(dtype):
    return TOL_F64 if dtype == torch.float64 else TOL_F32


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().double().cpu().numpy()


def image_case(ny, nx, seed, noise=0.05, polygons=20, dtype=np.float32):
    clean, noisy = synth.polygon_image(ny, nx, seed, polygons=polygons, noise=noise, dtype=dtype)
    return clean, noisy


def signal_case(n, seed, noise=0.1, dtype=np.float64):
    clean, noisy = synth.signal_1d(n, seed, noise=noise, min_len=min(16, max(1, n // 12)),
                                   segments=min(12, max(1, n // 16)), dtype=dtype)
    return clean, noisy


def make_pair(guide_np, radius, ss, sr, window="square", mode="onthefly", dtype=torch.float32):
    """(GPU graph, oracle graph) for the same guide; the oracle takes the guide as the GPU
    sees it (rounded to the GPU dtype).  For stored weights (FP32 or BF16) the oracle graph
    is built from the exported stored values, i.e. the exact operator of the stored graph
    (their rounding is checked separately against Eq. 2)."""
    g_dev = dev(guide_np, dtype)
    G = bf().bf_weights(g_dev, radius, ss, sr, window=window, weight_mode=mode)
    shape = (1, guide_np.size) if guide_np.ndim == 1 else guide_np.shape
    guide_seen = g_dev.double().cpu().numpy()
    if mode != "onthefly":
        taps = host(bf().graph_export_weights(G))
        O = Graph.from_taps(taps, shape, radius, window)
    else:
        O = Graph(guide_seen, shape, radius, ss, sr, window)
    return G, O

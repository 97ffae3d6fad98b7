"""Expected values of the 2048 x 2048 precision study, written by the FP64 oracle alone.

The workload is the 2048 x 2048 polygon image of seed 3 (noise 0.05) as the GPU sees it
(FP32 values), 7 x 7 window, sigma_s = 2, sigma_r = 0.08 (Eq. 2).
  * CG: 50 iterations (Algorithm 2, Jacobi), started from the noisy image.
  * Block LOBPCG: k = 32, 30 iterations (Algorithm 3, pencil (L, D), Jacobi), started
    from synth.block_start(noisy, 32, 3) (FP32 values).

It is run on two operators:
  * "exact": Eq. 2 weights in FP64.
  * "bf16": the operator whose weights are stored in BF16. Each FP64 weight is rounded to
    FP32, then to BF16 (nearest even), and the degree is summed from the rounded weights,
    so that operator is a graph in its own right.

Saved per operator: theta, the LOBPCG residual norms, the iteration and restart counts,
the CG output and the LOBPCG filtered signal y at 4096 sampled pixels, and the norms of
both outputs.

    OMP_NUM_THREADS=6 python tests/golden/make_precision_2048.py   # about an hour on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import solvers  # noqa: E402
from oracle.graph import Graph  # noqa: E402
from paper_1509_02468_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "precision_2048.npz")
NSAMPLE = 4096


def bf16_round(w64):
    """FP64 -> FP32 -> BF16 (round to nearest even on the upper 16 bits), as FP64."""
    w32 = np.asarray(w64, dtype=np.float32)
    bits = w32.view(np.uint32).astype(np.uint64)
    rb = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    return rb.astype(np.uint32).view(np.float32).astype(np.float64)


def run(tag, G, x0, X0, w, sample, out, log):
    t = time.time()
    cg = solvers.cg(G, x0, w.cg_iters)
    log(f"{tag}: CG {w.cg_iters} in {time.time() - t:.0f} s")
    t = time.time()
    lob = solvers.lobpcg(G, X0, w.lobpcg_iters)
    log(f"{tag}: LOBPCG k={X0.shape[1]} x {w.lobpcg_iters} in {time.time() - t:.0f} s, status {lob['status']}")
    out[f"{tag}_cg_x"] = cg["x"][sample]
    out[f"{tag}_cg_norm"] = np.linalg.norm(cg["x"])
    out[f"{tag}_theta"] = lob["theta"]
    out[f"{tag}_resid"] = lob["resid"]
    out[f"{tag}_y"] = lob["y"][sample]
    out[f"{tag}_y_norm"] = np.linalg.norm(lob["y"])
    out[f"{tag}_iters"] = lob["iters"]
    out[f"{tag}_restarts"] = lob["restarts"]


def main():
    log = lambda m: print(m, flush=True)
    w = synth.IMAGE_2048
    _, noisy = synth.make_input(w)
    ny, nx = noisy.shape
    x0 = noisy.astype(np.float64).reshape(-1)
    X0 = synth.block_start(noisy.reshape(-1), w.lobpcg_k, w.seed).astype(np.float64)
    sample = np.sort(np.random.default_rng(12345).choice(x0.size, NSAMPLE, replace=False))
    out = {"sample": sample, "shape": np.array([ny, nx]), "k": w.lobpcg_k,
           "lobpcg_iters": w.lobpcg_iters, "cg_iters": w.cg_iters}
    t = time.time()
    G = Graph(noisy.astype(np.float64), (ny, nx), w.radius, w.sigma_s, w.sigma_r)
    log(f"exact graph in {time.time() - t:.0f} s")
    taps_b = bf16_round(G.taps)
    run("exact", G, x0, X0, w, sample, out, log)
    del G
    t = time.time()
    Gb = Graph.from_taps(taps_b, (ny, nx), w.radius)
    del taps_b
    log(f"bf16 graph in {time.time() - t:.0f} s")
    run("bf16", Gb, x0, X0, w, sample, out, log)
    np.savez_compressed(OUT, **out)
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()

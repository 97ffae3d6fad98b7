"""Training and evaluation of the learned preconditioner (bf_net, include/bf.h).

Pairs (r, z): r is a residual that flexible CG with the Jacobi preconditioner produces on
the shifted system (L + sigma I) x = sigma x0 of a generated image (Algorithm 2 with the
shift of the Tikhonov graph filter), z solves (L + sigma I) z = r to a relative residual
of 1e-8 (FP64 CG on the GPU).  The net is trained on the loss ||T(r) - z||^2 / ||z||^2
with Adam, by the library's own forward and backward kernels, starting from weights with
which T is exactly Jacobi (D^-1).  Evaluation: iterations and time of flexible CG to a
relative residual of 1e-5 with the trained net against Jacobi, on held-out images.

The symmetric positive definite preconditioner (bf_spd, T = D^-1/2 (I + K^T K) D^-1/2) is
trained the same way by its own kernels, on pairs with white-noise r (make_random_pairs)
and the A-norm loss (z - T r)^T A (z - T r) / z^T A z (train_spd).

    python -m paper_1509_02468_gb300.train --images 200 --side 256 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import bf, synth

SIGMA = 1e-2
RADIUS, SIGMA_S, SIGMA_R = 3, 2.0, 0.08
CG_PICKS = (0, 1, 2, 4, 6, 9, 13, 19)          # residuals after these many iterations


def initial_weights(noise: float = 1e-2, seed: int = 0):
    """Jacobi-equivalent weights (channels 0/1 carry +-(D^-1 r)/rho through both ReLUs,
    layer 3 takes their difference) plus N(0, noise^2) elsewhere."""
    rng = np.random.default_rng(seed)
    W1 = noise * rng.standard_normal((16, 3, 3, 3))
    W2 = noise * rng.standard_normal((16, 16, 3, 3))
    W3 = noise * rng.standard_normal((1, 16, 3, 3))
    W1[0:2] = 0.0
    W1[0, 0, 1, 1], W1[1, 0, 1, 1] = 1.0, -1.0
    W2[0:2] = 0.0
    W2[0, 0, 1, 1], W2[1, 1, 1, 1] = 1.0, 1.0
    W3[0, 0:2] = 0.0
    W3[0, 0, 1, 1], W3[0, 1, 1, 1] = 1.0, -1.0
    return [W1.astype(np.float32), W2.astype(np.float32), W3.astype(np.float32)]


def make_pairs(seeds, side: int, sigma: float = SIGMA, picks=CG_PICKS, tol: float = 1e-8,
               kmax_solve: int = 20000, device="cuda"):
    """[(graph, r, z)] for the given image seeds (graphs kept alive with the pairs)."""
    out = []
    for s in seeds:
        _, noisy = synth.polygon_image(side, side, s)
        g32 = torch.as_tensor(noisy, device=device)
        G = bf.bf_weights(g32, RADIUS, SIGMA_S, SIGMA_R)
        G64 = bf.bf_weights(g32.double(), RADIUS, SIGMA_S, SIGMA_R)
        x0 = g32.reshape(-1).contiguous()
        for j in picks:
            x = x0.clone() if j == 0 else bf.cg_filter(G, x0, j, shift=sigma)[0]
            r = bf.shifted_residual(G, x0, x, sigma)
            z, info, _ = bf.cg_filter(G64, (r / sigma).double(), kmax_solve, shift=sigma, tol=tol)
            out.append((G, r.contiguous(), z.float().contiguous()))
    return out


def train(net, pairs, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    """Adam on mini-batches of pairs; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot, cnt = 0.0, 0
        lr_ep = lr * (0.5 ** (ep // max(1, epochs // 3)))
        for b0 in range(0, len(order), batch):
            idx = order[b0:b0 + batch]
            net.zero_grad()
            for i in idx:
                G, r, z = pairs[i]
                net.accumulate(G, r, z)
            _, loss = net.grad()
            tot += loss
            cnt += len(idx)
            net.adam(lr_ep, 1.0 / len(idx))
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.5f} (lr {lr_ep:.1e})")
    return hist


def make_random_pairs(seeds, side: int, per_image: int, sigma: float = SIGMA, tol: float = 1e-8,
                      kmax_solve: int = 20000, seed: int = 0, device="cuda"):
    """[(graph, r, z)]: per image, per_image residuals r ~ N(0, 1) on its grid (every
    frequency present) and z solving (L + sigma I) z = r to tol by FP64 CG on the GPU."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for s in seeds:
        _, noisy = synth.polygon_image(side, side, s)
        g32 = torch.as_tensor(noisy, device=device)
        G = bf.bf_weights(g32, RADIUS, SIGMA_S, SIGMA_R)
        G64 = bf.bf_weights(g32.double(), RADIUS, SIGMA_S, SIGMA_R)
        for _ in range(per_image):
            r = torch.randn(noisy.size, device=device, generator=gen)
            z, info, _ = bf.cg_filter(G64, (r / sigma).double(), kmax_solve, shift=sigma, tol=tol)
            out.append((G, r.contiguous(), z.float().contiguous()))
    return out


def spd_initial_kernel(half: int = 3, centre: float = 0.1, noise: float = 1e-2, seed: int = 0):
    """A small start for K (T = D^-1/2 (I + K^T K) D^-1/2 is then close to Jacobi); K = 0
    itself is a stationary point of the loss (T depends on K quadratically)."""
    rng = np.random.default_rng(seed)
    K = noise * rng.standard_normal((2 * half + 1, 2 * half + 1))
    K[half, half] += centre
    return K.astype(np.float32)


def train_spd(spd, pairs, epochs: int, lr: float, sigma: float = SIGMA, log=None):
    """Full-batch Adam on the A-norm loss of the SPD preconditioner (bf_spd_accumulate):
    one step per epoch on the mean gradient over all pairs; returns the mean loss of every
    epoch."""
    hist = []
    for ep in range(epochs):
        spd.zero_grad()
        for G, r, z in pairs:
            spd.accumulate(G, sigma, r, z)
        _, loss = spd.grad()
        hist.append(loss / max(len(pairs), 1))
        spd.adam(lr, 1.0 / max(len(pairs), 1))
        if log and ep % 50 == 0:
            log(f"epoch {ep}: mean A-norm loss {hist[-1]:.5f}")
    return hist


def mean_loss(net, pairs):
    tot = 0.0
    for G, r, z in pairs:
        net.zero_grad()
        net.accumulate(G, r, z)
        tot += net.grad()[1]
    net.zero_grad()
    return tot / max(len(pairs), 1)


def refined_cg(G32, G64, x0, sigma: float, tol: float, precond: str, net=None, inner_tol: float = 1e-3,
               inner_kmax: int = 3000, outer_max: int = 30, spd=None):
    """(L + sigma I) x = sigma x0 to a true relative residual tol by the library's
    mixed-precision refinement (cg_refine: FP64 residuals on G64, FP32 flexible CG on G32 to
    inner_tol).  Returns (x, rel, inner iterations, outer steps); rel is NaN when an inner
    solve broke down."""
    try:
        x, info = bf.cg_refine(G64, G32, x0.double().contiguous(), sigma, tol, precond=precond, net=net,
                               inner_tol=inner_tol, inner_kmax=inner_kmax, outer_max=outer_max, spd=spd)
    except bf.BFError:                          # breakdown or non-finite scalars: give up
        return x0.double(), float("nan"), 0, 0
    return x, info.rnorm / info.ref, info.iters, info.restarts


def evaluate(net, side: int, seed: int, sigma: float = SIGMA, tol: float = 1e-5, reps: int = 2,
             lob_k: int = 16, lob_iters: int = 30, device="cuda"):
    """Jacobi against the net on a held-out image: flexible CG to a true relative residual
    tol on (L + sigma I) x = sigma x0 (iterations, time, Mpix/s), and LOBPCG(k) for the
    pencil (L, D) after lob_iters steps (largest relative residual)."""
    _, noisy = synth.polygon_image(side, side, seed)
    g32 = torch.as_tensor(noisy, device=device)
    G = bf.bf_weights(g32, RADIUS, SIGMA_S, SIGMA_R)
    G64 = bf.bf_weights(g32.double(), RADIUS, SIGMA_S, SIGMA_R)
    x0 = g32.reshape(-1).contiguous()
    X0 = torch.as_tensor(synth.block_start(noisy.ravel(), lob_k, seed), device=device)
    res = {}
    for name, pc in (("jacobi", "jacobi"), ("net", "net")):
        kw = dict(precond=pc, net=net if pc == "net" else None)
        refined_cg(G, G64, x0, sigma, tol, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            x, rel, inner, outer = refined_cg(G, G64, x0, sigma, tol, **kw)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        lob = bf.lobpcg_filter(G, X0, lob_iters, **kw)
        res[name] = {"cg_inner_iters": inner, "cg_outer": outer, "cg_rel_residual": rel,
                     "cg_converged": bool(rel <= tol), "cg_seconds": dt, "cg_mpix_s": side * side / dt / 1e6,
                     "lobpcg_max_resid": float(lob["resid"].max()), "lobpcg_theta0": float(lob["theta"][0])}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--images", type=int, default=200)
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval-side", type=int, default=1024)
    ap.add_argument("--eval-seed", type=int, default=5)
    ap.add_argument("--out", default=None)
    ap.add_argument("--weights", default=None, help="evaluate these trained weights (.npz) only")
    a = ap.parse_args(argv)
    if a.weights:
        net = bf.Net(np.load(a.weights)["weights"])
        print(json.dumps({"eval": evaluate(net, a.eval_side, a.eval_seed),
                          "eval_jacobi_init": evaluate(bf.Net(initial_weights(noise=0.0)), a.eval_side, a.eval_seed),
                          "eval_image": f"{a.eval_side}x{a.eval_side} seed {a.eval_seed}"}))
        return
    t0 = time.time()
    pairs = make_pairs(range(a.seed0, a.seed0 + a.images), a.side)
    t_pairs = time.time() - t0
    net = bf.Net(initial_weights())
    loss0 = mean_loss(net, pairs)
    hist = train(net, pairs, a.epochs, a.batch, a.lr, log=print)
    ev = evaluate(net, a.eval_side, a.eval_seed)
    rep = {"images": a.images, "side": a.side, "pairs": len(pairs), "sigma": SIGMA,
           "seconds_pairs": t_pairs, "seconds_total": time.time() - t0,
           "loss_jacobi_init": loss0, "loss_per_epoch": hist, "eval": ev,
           "eval_image": f"{a.eval_side}x{a.eval_side} seed {a.eval_seed}"}
    print(json.dumps(rep))
    if a.out:
        np.savez(a.out, weights=net.weights(), report=json.dumps(rep))


if __name__ == "__main__":
    main()

"""The 2048 x 2048 precision study: the CG and LOBPCG filters (Algorithms 2 and 3) on the
GPU in each precision mode, against the FP64 oracle of the exact operator and of the
operator with BF16-stored weights.  The expected values at sampled pixels are in
tests/golden/precision_2048.npz, written by tests/golden/make_precision_2048.py from the
oracle alone.

Modes: weights computed on the fly in FP32 or stored in BF16; Gram products in FP32
(SIMT, FP64 folding), split-BF16 or BF16 on the tensor cores.  The bars: FP32 filter
outputs within 1e-5 (relative L2 over the sampled pixels) and Ritz values within 1e-6
(reading A8) of the oracle of the same operator; BF16 storage moves the operator itself
by about 2^-9 per weight, so against the exact oracle it is reported, not held to 1e-5;
BF16 Gram products (one product ~2^-8, split ~2^-16 relative per entry) move the Ritz
values by a few 1e-4 at this size: stated and bounded, not held to the FP32 bar."""
import os

import numpy as np
import pytest

from tests.gpu_helpers import TOL_F32, TOL_RITZ, bf, dev, host

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "precision_2048.npz")
MODES = [("onthefly", "fp32"), ("onthefly", "bf16x3"), ("onthefly", "bf16"), ("stored_bf16", "fp32")]
TABLE = {}


def ritz_err(th, ref):
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(np.asarray(th, np.float64) - ref) / scale))


def sample_err(v, ref):
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(np.asarray(v, np.float64) - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def case():
    if not os.path.exists(GOLD):
        pytest.skip("precision_2048.npz not generated")
    from paper_1509_02468_gb300 import synth
    gold = dict(np.load(GOLD))
    w = synth.IMAGE_2048
    _, noisy = synth.make_input(w)
    X0 = synth.block_start(noisy.reshape(-1), w.lobpcg_k, w.seed)
    yield gold, w, noisy, X0
    if TABLE:
        print("\nprecision study 2048x2048 (errors vs the FP64 oracle of the exact / BF16-stored operator)")
        for (wm, gr), e in TABLE.items():
            print(f"  weights {wm:12s} gram {gr:7s}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))


@pytest.mark.parametrize("wmode,gram", MODES)
def test_precision_mode(case, wmode, gram):
    gold, w, noisy, X0 = case
    s = gold["sample"]
    G = bf().bf_weights(dev(noisy), w.radius, w.sigma_s, w.sigma_r, weight_mode=wmode)
    x, info, _ = bf().cg_filter(G, dev(noisy.reshape(-1)), w.cg_iters)
    out = bf().lobpcg_filter(G, dev(X0), w.lobpcg_iters, gram=gram, want_X=False)
    xs, ys = host(x)[s], host(out["y"])[s]
    th = host(out["theta"])
    e = {}
    for tag in ("exact", "bf16"):
        e[f"theta[{tag}]"] = ritz_err(th, gold[f"{tag}_theta"])
        e[f"y[{tag}]"] = sample_err(ys, gold[f"{tag}_y"])
        e[f"cg[{tag}]"] = sample_err(xs, gold[f"{tag}_cg_x"])
    TABLE[(wmode, gram)] = e
    assert np.all(np.isfinite(th)) and np.all(np.isfinite(ys))
    own = "exact" if wmode == "onthefly" else "bf16"
    # CG does not use the Gram: FP32 on either operator meets the FP32 bar
    assert e[f"cg[{own}]"] <= TOL_F32, e
    if gram == "fp32":
        assert e[f"theta[{own}]"] <= TOL_RITZ, e
        assert e[f"y[{own}]"] <= TOL_F32, e
    else:
        # BF16 Gram products (split: hi*hi + hi*lo + lo*hi, ~2^-16 relative per entry; plain:
        # ~2^-8) perturb the Rayleigh-Ritz pencil; here that moves the Ritz values and y by a
        # few 1e-4 (measured 1.7e-4 / 2.3e-4 split, 4.5e-4 / 2.1e-4 plain): reported, with a
        # bound, not held to the FP32 bar
        assert e[f"theta[{own}]"] <= 2e-3, e
        assert e[f"y[{own}]"] <= 2e-3, e
    if wmode == "stored_bf16":
        # the stored operator differs from the exact one by the BF16 rounding of its weights
        assert e["cg[exact]"] <= 2.0 ** -6, e

"""The image experiment of Section 7 on the GPU: the 5-point lattice (cross window of
radius 1) with bilateral weights of range width sigma_r = 0.1 (the spatial factor is 1 on
a lattice: sigma_s = inf), noise of variance 0.01, and 20 iterations of CG (Algorithm 2)
and of LOBPCG (Algorithm 3) with and without the constraint x _|_ e, each against the FP64
oracle."""
import math

import numpy as np
import pytest

from oracle import solvers
from paper_1509_02468_gb300 import synth
from tests.gpu_helpers import TOL_F32, TOL_RITZ, bf, dev, host, make_pair, rel_l2

pytestmark = pytest.mark.gpu

SIDE, SIGMA_R, ITERS = 256, 0.1, 20


def _image():
    _, noisy = synth.polygon_image(SIDE, SIDE, 71, noise=0.1)
    return noisy


def _ritz_err(theta, ref):
    floor = 1e-3 * np.abs(ref).max()
    return float(np.max(np.abs(theta - ref) / np.maximum(np.abs(ref), floor)))


def test_lattice_apply_all_ops():
    g = _image()
    G, O = make_pair(g, 1, math.inf, SIGMA_R, window="cross")
    X = np.random.default_rng(1).standard_normal((g.size, 4)).astype(np.float32)
    for op in ("W", "L", "DINV_W", "D", "NSYM", "NDIAGL"):
        Y = host(bf().bf_apply(G, op, dev(X)))
        assert rel_l2(Y, O.apply(op, X.astype(np.float64))) <= TOL_F32, op


def test_lattice_cg_20():
    g = _image()
    G, O = make_pair(g, 1, math.inf, SIGMA_R, window="cross")
    x, info, h = bf().cg_filter(G, dev(g.reshape(-1)), ITERS, hist=True)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), ITERS)
    assert info.iters == ref["iters"] == ITERS
    assert rel_l2(host(x), ref["x"]) <= TOL_F32
    np.testing.assert_allclose(host(h).reshape(-1, 2)[:, 0], ref["alpha"], rtol=1e-5)


@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("constrain", [False, True])
def test_lattice_lobpcg_20(k, constrain):
    g = _image()
    G, O = make_pair(g, 1, math.inf, SIGMA_R, window="cross")
    X0 = synth.block_start(g.reshape(-1), k, seed=71)
    X0d = dev(X0)
    out = bf().lobpcg_filter(G, X0d, ITERS, constrain=constrain)
    ref = solvers.lobpcg(O, host(X0d), ITERS, constrain=constrain)
    assert out["info"].iters == ref["iters"] == ITERS
    assert _ritz_err(host(out["theta"]), ref["theta"]) <= TOL_RITZ
    assert rel_l2(host(out["y"]), ref["y"]) <= TOL_F32

"""Batched CG (bf_batch: one work list over many uneven instances, one CUDA graph) against
the FP64 oracle per instance and against the single-instance GPU path."""
import numpy as np
import pytest
import torch

from oracle import solvers
from tests.gpu_helpers import TOL_F32, bf, dev, host, image_case, make_pair, rel_l2, signal_case

pytestmark = pytest.mark.gpu


def mixed(seed=0):
    """Images of ragged sizes (7x7 window), signals (11 taps) and one 5-point-lattice image."""
    cases = []
    for (ny, nx) in [(40, 37), (64, 64), (17, 100), (9, 9)]:
        _, noisy = image_case(ny, nx, seed + ny)
        G, O = make_pair(noisy, 3, 2.0, 0.08)
        cases.append((G, O, noisy.ravel()))
    for n in (500, 1234):
        _, noisy = signal_case(n, seed + n, dtype=np.float32)
        G, O = make_pair(noisy, 5, 3.0, 0.1)
        cases.append((G, O, noisy.ravel()))
    _, noisy = image_case(30, 33, seed + 7)
    G, O = make_pair(noisy, 1, 2.0, 0.1, window="cross")
    cases.append((G, O, noisy.ravel()))
    return cases


@pytest.mark.parametrize("shift", [0.0, 1e-2])
def test_batched_cg_matches_oracle_and_single_path(shift):
    cases = mixed()
    B = bf().Batch([c[0] for c in cases])
    x0s = [dev(c[2]) for c in cases]
    outs, infos = B.cg(x0s, 12, shift=shift)
    for (G, O, x0), x, info in zip(cases, outs, infos):
        ref = solvers.cg(O, x0.astype(np.float64), 12, shift=shift)
        assert info.iters == ref["iters"]
        assert rel_l2(host(x), ref["x"]) <= TOL_F32
        single, sinfo, _ = bf().cg_filter(G, dev(x0), 12, shift=shift)
        assert rel_l2(host(x), host(single)) <= 1e-6
        assert sinfo.iters == info.iters


def test_batched_cg_with_tolerance_stops_each_instance():
    cases = mixed(seed=3)
    B = bf().Batch([c[0] for c in cases])
    x0s = [dev(c[2]) for c in cases]
    outs, infos = B.cg(x0s, 200, shift=1e-1, tol=1e-4)
    for (G, O, x0), x, info in zip(cases, outs, infos):
        single, sinfo, _ = bf().cg_filter(G, dev(x0), 200, shift=1e-1, tol=1e-4)
        assert info.status == sinfo.status == "converged"
        assert info.iters == sinfo.iters
        assert rel_l2(host(x), host(single)) <= 1e-6


def test_graph_replay_and_autotune_keep_results():
    cases = mixed(seed=5)
    B = bf().Batch([c[0] for c in cases])
    x0s = [dev(c[2]) for c in cases]
    first, _ = B.cg(x0s, 8)
    x0b = [x * 0.5 + 0.25 for x in x0s]
    second, _ = B.cg(x0b, 8)                 # replay of the captured graph, new inputs
    for (G, O, x0), x in zip(cases, second):
        ref = solvers.cg(O, 0.5 * x0.astype(np.float64) + 0.25, 8)
        assert rel_l2(host(x), ref["x"]) <= TOL_F32
    ms = B.tune(x0s, iters=3)
    assert len(ms) == 3 and all(m > 0 for m in ms)
    tiles, variant = B.tiles()
    assert variant == int(np.argmin(ms)) and tiles > 0
    tuned, _ = B.cg(x0s, 8)
    for a, b in zip(first, tuned):
        assert rel_l2(host(b), host(a)) <= 1e-6


def test_batch_rejects_unsupported_graphs():
    _, noisy = image_case(16, 16, 1)
    G64 = bf().bf_weights(dev(noisy, torch.float64), 3, 2.0, 0.08)
    with pytest.raises(bf().BFError):
        bf().Batch([G64])
    Ga = bf().bf_weights(dev(noisy), 3, 2.0, 0.08)
    Gb = bf().bf_weights(dev(noisy), 3, 2.5, 0.08)
    with pytest.raises(bf().BFError):
        bf().Batch([Ga, Gb])
    Gs = bf().bf_weights(dev(noisy), 3, 2.0, 0.08, weight_mode="stored_f32")
    with pytest.raises(bf().BFError):
        bf().Batch([Gs])


@pytest.mark.parametrize("shift,tol", [(0.0, 0.0), (1e-2, 0.0), (1e-1, 1e-4)])
def test_persistent_run_equals_graph_run(shift, tol):
    """One cooperative launch with grid barriers gives the per-phase run's results exactly
    (same jobs, same reduction order) and matches the oracle."""
    cases = mixed(seed=7)
    B = bf().Batch([c[0] for c in cases])
    x0s = [dev(c[2]) for c in cases]
    kmax = 200 if tol > 0 else 12
    outs_g, infos_g = B.cg(x0s, kmax, shift=shift, tol=tol)
    outs_p, infos_p = B.cg_persistent(x0s, kmax, shift=shift, tol=tol)
    for (G, O, x0), xg, xp, ig, ip in zip(cases, outs_g, outs_p, infos_g, infos_p):
        assert torch.equal(xg, xp)
        assert ig.iters == ip.iters and ig.status == ip.status
        if tol == 0.0:
            ref = solvers.cg(O, x0.astype(np.float64), kmax, shift=shift)
            assert rel_l2(host(xp), ref["x"]) <= TOL_F32


def test_persistent_barrier_wait_gives_up_and_context_survives():
    """A CTA that never reaches the first grid barrier: every other CTA's bounded wait runs
    out (1 s), the call reports BF_ETIMEOUT, and the next run on the same batch is right."""
    cases = mixed(seed=9)
    B = bf().Batch([c[0] for c in cases])
    x0s = [dev(c[2]) for c in cases]
    with pytest.raises(bf().BFError) as ei:
        B.barrier_test(x0s, kmax=3)
    assert ei.value.code == bf().BF_ETIMEOUT
    outs, infos = B.cg_persistent(x0s, 8)
    for (G, O, x0), x, info in zip(cases, outs, infos):
        ref = solvers.cg(O, x0.astype(np.float64), 8)
        assert info.iters == 8
        assert rel_l2(host(x), ref["x"]) <= TOL_F32


def test_batched_lobpcg_equals_single_calls_and_oracle():
    """Algorithm 3 on every instance over a pool of streams: each instance's Ritz values and
    filtered signal equal those of its own lobpcg_filter call exactly, and the oracle's."""
    from paper_1509_02468_gb300 import synth
    from tests.gpu_helpers import TOL_RITZ_SMALL_F32
    cases = mixed(seed=11)
    B = bf().Batch([c[0] for c in cases])
    k, kmax = 4, 10
    X0s = [dev(synth.block_start(c[2], k, seed=11 + i)) for i, c in enumerate(cases)]
    thetas, ys, infos = B.lobpcg(X0s, kmax, nstreams=3)
    for (G, O, x0), X0, th, y, info in zip(cases, X0s, thetas, ys, infos):
        single = bf().lobpcg_filter(G, X0, kmax, want_X=False)
        assert torch.equal(th, single["theta"]) and torch.equal(y, single["y"])
        assert info.iters == kmax
        ref = solvers.lobpcg(O, host(X0), kmax)
        scale = np.maximum(np.abs(ref["theta"]), 1e-3 * np.abs(ref["theta"]).max())
        assert np.max(np.abs(host(th) - ref["theta"]) / scale) <= TOL_RITZ_SMALL_F32
        assert rel_l2(host(y), ref["y"]) <= TOL_F32          # measured <= 7.5e-7

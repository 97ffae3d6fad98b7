"""The accuracy keys of the benchmark line (host logic, CPU): `err` compares the timed
step's outputs with the oracle's step, and `batched.err` the batched forms' CG outputs with
the oracle's CG on the smallest instances of the 256-instance batch."""
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_step_errors_relative_l2_and_ritz_floor():
    import bench
    rng = np.random.default_rng(0)
    ref = {"x_cg": rng.standard_normal(100), "y": rng.standard_normal(100),
           "theta": np.array([1e-9, 1e-3, 0.5, 1.0])}
    e = bench.step_errors(ref, ref["x_cg"] * (1 + 1e-6), ref["y"] + 1e-7 * np.linalg.norm(ref["y"]) * np.eye(100)[0],
                          ref["theta"] + np.array([1e-9, 0.0, 0.0, 0.0]))
    assert e["cg_x"] == pytest.approx(1e-6, rel=1e-6)
    assert e["lobpcg_y"] == pytest.approx(1e-7, rel=1e-6)
    # theta_0 = 1e-9 sits below the floor 1e-3 * theta_max: its error counts against 1e-3
    assert e["theta"] == pytest.approx(1e-9 / 1e-3, rel=1e-9)


def test_batch_oracle_errors_zero_for_the_oracle_and_picks_both_kinds():
    import bench
    from oracle import solvers
    from oracle.graph import Graph
    inst = bench._batch_inputs()
    assert len(inst) == 256 and {nd for nd, _ in inst} == {1, 2}
    # give every instance the oracle's own CG output: the reported error is FP32 rounding
    outs = [torch.zeros(1)] * len(inst)
    for nd in (1, 2):
        for i in sorted((i for i in range(len(inst)) if inst[i][0] == nd), key=lambda i: inst[i][1].size)[:4]:
            a = inst[i][1]
            g64 = np.asarray(a, np.float32).astype(np.float64)
            shape = a.shape if nd == 2 else (1, a.size)
            r, ss, sr = (3, 2.0, 0.08) if nd == 2 else (5, 3.0, 0.1)
            outs[i] = torch.as_tensor(solvers.cg(Graph(g64, shape, r, ss, sr), g64.reshape(-1), 50)["x"]).float()
    worst = bench._batch_oracle_errors(inst, {"exact": outs}, 50)
    assert worst["exact"] < 1e-7
    # a wrong output on one of the compared instances shows
    bad = list(outs)
    i_img = min((i for i in range(len(inst)) if inst[i][0] == 2), key=lambda i: inst[i][1].size)
    bad[i_img] = torch.as_tensor(inst[i_img][1].reshape(-1))          # the unfiltered input
    assert bench._batch_oracle_errors(inst, {"bad": bad}, 50)["bad"] > 1e-3

"""Plant plausible mistakes in a copy of the oracle and check that its pins catch each one.

Each case copies ``oracle/`` and the pin tests into a temporary directory, applies one
edit (a dropped factor, a wrong sign, a swapped index, a transposed operand, the wrong
matrix) and runs the pin tests there: they must fail.  The real oracle is never touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    # Eq. 2: spatial and range factors, window offsets
    ("oracle/graph.py", "(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s)",
     "(dx * dx + dy * dy) / (sigma_s * sigma_s)"),
    ("oracle/graph.py", "(2.0 * sigma_r * sigma_r)", "(sigma_r * sigma_r)"),
    ("oracle/graph.py", "ty, tx = yy + dy, xx + dx", "ty, tx = yy + dx, xx + dy"),
    # Eq. 4 and the normalised forms of Section 4
    ("oracle/graph.py", "self.L = (self.D - self.W).tocsr()", "self.L = (self.W - self.D).tocsr()"),
    ("oracle/graph.py", "dis = 1.0 / np.sqrt(self.d)", "dis = 1.0 / self.d"),
    ("oracle/graph.py", "self.diagL = np.bincount(rows[off], weights=vals[off], minlength=n)",
     "self.diagL = self.d.copy()"),
    # Algorithm 2
    ("oracle/solvers.py", "bk = num / den", "bk = -num / den"),
    ("oracle/solvers.py", "den = (s_old @ r_old) if beta == \"sr\" else (s_old @ s_old)",
     "den = (s_old @ s_old) if beta == \"sr\" else (s_old @ r_old)"),
    ("oracle/solvers.py", "r = r - a * q", "r = r + a * q"),
    ("oracle/solvers.py", "a = sr / pq", "a = sr / (p @ p)"),
    # Algorithm 3
    ("oracle/solvers.py", "R = AX - B(X) * theta[None, :]\n        if tol",
     "R = AX - X * theta[None, :]\n        if tol"),
    ("oracle/solvers.py", "P = S[:, k:] @ C[k:, :]", "P = S[:, :k] @ C[:k, :]"),
    ("oracle/solvers.py", "y = X @ (X.T @ (bdiag * x0v))", "y = X @ (X.T @ x0v)"),
    ("oracle/solvers.py", "return V - np.outer(e, (e @ B(V)) / eBe)",
     "return V - np.outer(e, (e @ V) / eBe)"),
    ("oracle/solvers.py", "C = C * s[:, None]", "C = C / s[:, None]"),
    # Section 4 simple iteration, Section 5 polynomial recurrence
    ("oracle/solvers.py", "x = G.DINV_W @ x", "x = G.W @ x"),
    ("oracle/spectral.py", "chi = chi + a * pi", "chi = chi + a * sig"),
    # Section 2's nonlinear iteration: guided by x0 instead of the iterate; a step without D^-1
    ("oracle/solvers.py", "G = Graph(x, shape, radius, sigma_s, sigma_r, window=window)",
     "G = Graph(x0, shape, radius, sigma_s, sigma_r, window=window)"),
    ("oracle/solvers.py", "window=window)\n        x = G.DINV_W @ x", "window=window)\n        x = x - G.L @ x"),
    # Section 3's guided filter: Algorithm 1 and the matrix of Eq. 6
    ("oracle/guided.py", "m11 = G2 + N * eps", "m11 = G2 + eps"),
    ("oracle/guided.py", "icpt = (m11 * X1 - G1 * GX) / det", "icpt = (m11 * X1 + G1 * GX) / det"),
    ("oracle/guided.py", "return (slope_sum * g + icpt_sum) / nwin", "return (slope_sum * x + icpt_sum) / nwin"),
    ("oracle/guided.py", "slope = (GX * N - G1 * X1) / det", "slope = (GX * N - G1 * X1) / (m11 * N)"),
    ("oracle/guided.py", "block = (1.0 + np.outer(dev, dev) / (var + eps)) / nk",
     "block = (1.0 + np.outer(dev, dev) / (var + eps)) / nk ** 2"),
    ("oracle/guided.py", "acc[ys0:ys1, xs0:xs1] += V[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]",
     "acc[ys0:ys1, xs0:xs1] += V[ys0 - dy:ys1 - dy, xs0 - dx:xs1 - dx]"),
    # the conv-net preconditioner: input scaling, adjoint shift, ReLU mask of the wrong layer
    ("oracle/convnet.py", "c0 = np.asarray(r, np.float64) / np.asarray(d, np.float64)",
     "c0 = np.asarray(r, np.float64)"),
    ("oracle/convnet.py", "shifted = gp[:, 1 - a:1 - a + H, 1 - b:1 - b + W]",
     "shifted = gp[:, 1 + a:1 + a + H, 1 + b:1 + b + W]"),
    ("oracle/convnet.py", 'G1 = conv_t(G2, W2) * (c["A1"] > 0)', 'G1 = conv_t(G2, W2) * (c["A2"] > 0)'),
    ("oracle/convnet.py", "vv = b2 * vv + (1 - b2) * g * g", "vv = b2 * vv + (1 - b2) * g"),
    # Adam's bias corrections without the step exponent (equal to the right ones at t = 1)
    ("oracle/convnet.py", "mh = mm / (1 - b1 ** t)", "mh = mm / (1 - b1)"),
    ("oracle/convnet.py", "vh = vv / (1 - b2 ** t)", "vh = vv / (1 - b2)"),
    # the symmetric positive definite T: transposed kernel, adjoint without the turn, the
    # outer D^-1/2 dropped, the loss gradient's sign and its second term
    ("oracle/precond_spd.py", "y[i0:i1, j0:j1] += K[a + h, b + h] *", "y[i0:i1, j0:j1] += K[b + h, a + h] *"),
    ("oracle/precond_spd.py", "return correlate(y, np.asarray(K)[::-1, ::-1])", "return correlate(y, np.asarray(K))"),
    ("oracle/precond_spd.py", "return dh * t.reshape(-1)", "return t.reshape(-1)"),
    ("oracle/precond_spd.py", "hv = (dh * (-2.0 * Ae / c))", "hv = (dh * (2.0 * Ae / c))"),
    ("oracle/precond_spd.py", "grad[a + hk, b + hk] = s1 + s2", "grad[a + hk, b + hk] = s1"),
]


@pytest.mark.parametrize("path,old,new", MUTATIONS, ids=[f"{m[0].split('/')[-1]}:{i}" for i, m in enumerate(MUTATIONS)])
def test_pins_catch_planted_mistake(tmp_path, path, old, new):
    for sub in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "test_oracle_mutations.py"))
    shutil.copytree(os.path.join(ROOT, "paper_1509_02468_gb300"), tmp_path / "paper_1509_02468_gb300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "csrc"))
    target = tmp_path / path
    src = target.read_text()
    assert old in src, f"mutation anchor not found in {path}: {old!r}"
    target.write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_precond_spd.py", "tests/test_oracle_graph.py",
                        "tests/test_oracle_solvers.py", "tests/test_oracle_convnet.py",
                        "tests/test_oracle_guided.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake not caught: {path}: {new!r}\n{r.stdout[-2000:]}"

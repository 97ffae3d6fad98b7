"""Oracle: the filters of Sections 4-6 run on explicit FP64 matrices.

Test infrastructure only (see ``oracle/__init__``).

* ``simple_iteration`` -- x_{k+1} = D^-1 W x_k = x_k - D^-1 L x_k (Section 4, Eq. 3).
* ``reguided_iteration`` -- the nonlinear iteration of Section 2: the weights are rebuilt
                          from each iterate, x_{k+1} = D(x_k)^-1 W(x_k) x_k.
* ``cg``               -- Algorithm 2: preconditioned CG for L x = 0 started at x0, with the
                          flexible beta of Section 5; optionally the shifted system
                          (L + sigma I) x = sigma x0 (a Tikhonov graph filter) and a
                          residual tolerance.
* ``lobpcg``           -- Algorithm 3 for a block of k vectors: Rayleigh-Ritz for the pencil
                          (L, B), B = D (or I), on span{X, W, P} with W = T(L X - B X Theta),
                          optionally constrained B-orthogonal to the constant vector e.

Readings of the text where it leaves a choice, each with its reason:
* beta.  Algorithm 2 prints beta = s^T (r - r_old) / (s_old^T s_old).  Its denominator is
  consistent with the numerator of alpha (s^T r) only when the preconditioner is the
  identity; the flexible (Polak-Ribiere) CG of the works it cites divides by
  s_old^T r_old.  ``beta="sr"`` (default) uses s_old^T r_old; ``beta="ss"`` is the printed
  formula.  They coincide when T = I.
* stopping.  The loop ends early when s^T r = 0 (the exact solution was reached) or when
  p^T q <= 0 (breakdown; x is left as it was).  With ``tol`` > 0 it also ends once
  ||r|| <= tol * ||b|| (||r_0|| when b = 0).
* LOBPCG output.  The Ritz vectors are normalised X^T B X = I (Algorithm 3 fixes the
  coefficient of w instead, which leaves the amplitude free).  The filtered signal is the
  B-orthogonal projection of x0 on span(X): y = X X^T B x0; with the constraint the
  B-mean e_bar = e^T B x0 / e^T B e is added back: y = e_bar e + X X^T B (x0 - e_bar e).
* LOBPCG start.  Algorithm 3 is stated for one vector started at x0: in a block, column 0
  is x0 and the other columns are given by the caller.
* LOBPCG search direction.  Algorithm 3 sets p_k+1 = w_k + gamma_k p_k.  For a block the
  raw P drifts into span X as columns converge and S^T B S becomes ill-conditioned; P is
  therefore kept B-orthogonal to X after each update (the same trial subspaces, see
  ``lobpcg``), as in the basis selection of Hetmaniuk and Lehoucq (2006).
* Rayleigh-Ritz.  The small pencil (S^T A S, S^T B S) is scaled to unit diagonal, reduced
  with the Cholesky factor of the scaled S^T B S, solved as a symmetric eigenproblem and
  sorted ascending.  If that Cholesky factor has a squared pivot <= ``DEP_TOL`` (the
  trial basis is numerically dependent), the iteration is redone without P; if it still
  fails the run stops with status "breakdown".
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .graph import Graph

DEP_TOL = 1e-10


# ---------------------------------------------------------------- simple iteration (Section 4)
def simple_iteration(G, x0, iters: int):
    """iters BF steps with fixed weights: x <- D^-1 W x (Eq. 3)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    for _ in range(iters):
        x = G.DINV_W @ x
    return x


def reguided_iteration(x0, shape, radius: int, sigma_s: float, sigma_r: float, iters: int,
                       window: str = "square"):
    """iters BF steps that change the weights every step (Section 2, the first of the two
    ways to iterate the filter): the graph of Eq. 2 is built from the current iterate as
    guide, then one step x <- D(x)^-1 W(x) x is taken.  A nonlinear filter: no fixed
    Laplacian describes the whole cascade."""
    x = np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    for _ in range(iters):
        G = Graph(x, shape, radius, sigma_s, sigma_r, window=window)
        x = G.DINV_W @ x
    return x


# ---------------------------------------------------------------- preconditioners
def make_precond(G, kind="jacobi"):
    """T as a function of a vector or block: 'jacobi' = D^-1 (Algorithm 2), 'identity' = I,
    or any callable."""
    if callable(kind):
        return kind
    if kind == "jacobi":
        dinv = 1.0 / G.d
        return lambda r: (dinv * r.T).T
    if kind == "identity":
        return lambda r: r.copy()
    raise ValueError(kind)


# ---------------------------------------------------------------- Algorithm 2
def cg(G, x0, kmax: int, precond="jacobi", beta: str = "sr", shift: float = 0.0,
       tol: float = 0.0):
    """Preconditioned CG(kmax) for A x = b with A = L + shift*I and b = shift*x0
    (shift = 0: Algorithm 2's L x = 0), started at x = x0.

    Returns a dict with x, the alpha and beta of every completed iteration (beta_1 = 0),
    the residual norms ||r|| after each iteration, the number of iterations done and a
    status string."""
    T = make_precond(G, precond)
    x0 = np.asarray(x0, dtype=np.float64)
    A = G.L if shift == 0.0 else (G.L + shift * sp.identity(G.n, format="csr")).tocsr()
    b = shift * x0
    x = x0.copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    ref = bnorm if bnorm > 0 else np.linalg.norm(r)
    alphas, betas, rnorms = [], [], []
    status = "ok"
    p = s_old = r_old = None
    for k in range(1, kmax + 1):
        s = T(r)
        if k == 1:
            bk = 0.0
            p_new = s.copy()
        else:
            num = s @ (r - r_old)
            den = (s_old @ r_old) if beta == "sr" else (s_old @ s_old)
            bk = num / den
            p_new = s + bk * p
        q = A @ p_new
        sr = s @ r
        pq = p_new @ q
        if sr == 0.0:
            status = "converged"
            break
        if not (pq > 0.0):
            status = "breakdown"
            break
        p = p_new
        a = sr / pq
        alphas.append(a)
        betas.append(bk)
        x = x + a * p
        r_old, s_old = r, s
        r = r - a * q
        rn = np.linalg.norm(r)
        rnorms.append(rn)
        if tol > 0.0 and rn <= tol * ref:
            status = "converged"
            break
    return {"x": x, "alpha": np.array(alphas), "beta": np.array(betas),
            "rnorm": np.array(rnorms), "iters": len(alphas), "status": status, "ref": ref}


# ---------------------------------------------------------------- Rayleigh-Ritz
def rayleigh_ritz(GA, GB, k):
    """k smallest eigenpairs of the pencil (GA, GB) (both symmetric, GB positive definite).

    Returns (theta, C, min_pivot2) with C^T GB C = I, or raises np.linalg.LinAlgError when
    the scaled GB is numerically singular (a squared Cholesky pivot <= DEP_TOL)."""
    GA = 0.5 * (GA + GA.T)
    GB = 0.5 * (GB + GB.T)
    dg = np.diag(GB)
    if np.any(~(dg > 0)):
        raise np.linalg.LinAlgError("non-positive diagonal in S^T B S")
    s = 1.0 / np.sqrt(dg)
    A1 = GA * s[:, None] * s[None, :]
    B1 = GB * s[:, None] * s[None, :]
    try:
        R = np.linalg.cholesky(B1)           # B1 = R R^T, R lower
    except np.linalg.LinAlgError:
        raise
    piv2 = np.diag(R) ** 2
    if piv2.min() <= DEP_TOL:
        raise np.linalg.LinAlgError(f"dependent trial basis (pivot^2 {piv2.min():.3e})")
    Y = sla.solve_triangular(R, A1, lower=True)            # R^-1 A1
    M = sla.solve_triangular(R, Y.T, lower=True).T          # R^-1 A1 R^-T
    M = 0.5 * (M + M.T)
    lam, V = np.linalg.eigh(M)
    order = np.argsort(lam, kind="stable")
    lam, V = lam[order], V[:, order]
    C = sla.solve_triangular(R.T, V[:, :k], lower=False)    # R^-T V
    C = C * s[:, None]
    return lam[:k].copy(), C, float(piv2.min())


# ---------------------------------------------------------------- Algorithm 3 (block)
def lobpcg(G, X0, kmax: int, pencil: str = "D", precond="jacobi", constrain: bool = False,
           tol: float = 0.0, x0=None, p_ortho: bool = True):
    """Block LOBPCG as a low-pass filter (Algorithm 3 with a block of k vectors).

    A = L, B = D (pencil "D") or I (pencil "I").  Returns a dict with theta (k Ritz values,
    ascending), X (B-orthonormal Ritz vectors [n][k]), resid (||L x_j - theta_j B x_j|| /
    ||B x_j||), y (the filtered signal), the Ritz values of every iteration, the number of
    iterations, the number of restarts without P and a status string.

    p_ortho: after every update P is made B-orthogonal to the new X (P -= X X^T B P).
    A X and A P are recomputed with the operator after every update (not carried as
    linear combinations), so S^T A S is always consistent with the vectors in S.
    span{X_t+1, P_t+1} = span{X_t+1, X_t} either way, so every trial subspace -- and hence
    every Ritz pair -- is the same as with the raw P = [W P] C_WP; only the conditioning of
    S^T B S changes (raw P drifts into span X as columns converge)."""
    L = G.L
    n = G.n
    bdiag = G.d.copy() if pencil == "D" else np.ones(n)
    T = make_precond(G, precond)
    X = np.array(X0, dtype=np.float64, copy=True).reshape(n, -1)
    k = X.shape[1]
    x0v = X[:, 0].copy() if x0 is None else np.asarray(x0, dtype=np.float64)
    e = np.ones(n)
    eBe = float(e @ (bdiag * e))

    def B(V):
        return bdiag[:, None] * V

    def proj(V):                    # B-orthogonal projection off e
        return V - np.outer(e, (e @ B(V)) / eBe)

    def borth(V):                   # Cholesky QR in the B inner product
        Gm = V.T @ B(V)
        R = np.linalg.cholesky(0.5 * (Gm + Gm.T))
        return sla.solve_triangular(R, V.T, lower=True).T

    if constrain:
        X = proj(X)
    X = borth(borth(X))
    AX = np.asarray(L @ X)
    theta, C, _ = rayleigh_ritz(X.T @ AX, X.T @ B(X), k)
    X = X @ C
    AX = AX @ C
    P = AP = None
    hist = [theta.copy()]
    restarts = 0
    status = "ok"
    it = 0
    for _ in range(kmax):
        R = AX - B(X) * theta[None, :]
        if tol > 0.0:
            res = np.linalg.norm(R, axis=0) / np.linalg.norm(B(X), axis=0)
            if res.max() <= tol:
                status = "converged"
                break
        W = T(R)
        if constrain:
            W = proj(W)
        AW = np.asarray(L @ W)
        use_p = P is not None
        while True:
            if use_p:
                S = np.hstack([X, W, P])
                AS = np.hstack([AX, AW, AP])
            else:
                S = np.hstack([X, W])
                AS = np.hstack([AX, AW])
            try:
                theta_new, C, _ = rayleigh_ritz(S.T @ AS, S.T @ B(S), k)
                break
            except np.linalg.LinAlgError:
                if use_p:
                    use_p = False
                    restarts += 1
                    continue
                status = "breakdown"
                theta_new = None
                break
        if theta_new is None:
            break
        theta = theta_new
        X = S @ C
        P = S[:, k:] @ C[k:, :]
        if p_ortho:
            P = P - X @ (X.T @ B(P))
        AX = np.asarray(L @ X)        # products with A are always fresh operator applies
        AP = np.asarray(L @ P)
        it += 1
        hist.append(theta.copy())
    R = AX - B(X) * theta[None, :]
    resid = np.linalg.norm(R, axis=0) / np.linalg.norm(B(X), axis=0)
    if constrain:
        ebar = float(e @ (bdiag * x0v)) / eBe
        y = ebar * e + X @ (X.T @ (bdiag * (x0v - ebar * e)))
    else:
        y = X @ (X.T @ (bdiag * x0v))
    return {"theta": theta, "X": X, "AX": AX, "resid": resid, "y": y,
            "theta_hist": np.array(hist), "iters": it, "restarts": restarts,
            "status": status}

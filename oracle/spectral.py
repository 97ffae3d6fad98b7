"""Oracle: dense spectral tools for small graphs (Section 4, Eq. 8; Section 5).

Test infrastructure only (see ``oracle/__init__``).  Used as pins on tiny inputs:

* ``pencil_eig``        -- all eigenpairs of L u = lambda B u (B = D or I) by a dense
                           symmetric eigensolver (Eq. 8 for B = I).
* ``cg_polynomial``     -- the polynomial chi_k with x_k = chi_k(D^-1 A) x0 built from the
                           alpha/beta that CG produced (Section 5: CG iterates are polynomial
                           filters of the preconditioned matrix).
* ``spectral_filter``   -- h(D^-1 A) x0 evaluated through the eigendecomposition of
                           D^-1/2 A D^-1/2: the vertex-domain filter seen in the graph
                           Fourier basis.
* ``lowpass_projection``-- the B-orthogonal projection of x0 on the k lowest eigenvectors.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pencil_eig(G, pencil: str = "D", op: str = "L"):
    """Eigenvalues (ascending) and B-orthonormal eigenvectors of (op, B), dense."""
    A = G.dense(op)
    if pencil == "D":
        return sla.eigh(A, np.diag(G.d))
    return np.linalg.eigh(A)


def cg_polynomial(alphas, betas, lam):
    """chi_k(lam) for the CG run with the given alpha_j, beta_j (beta_1 unused).

    With s = D^-1 r the CG updates x += a p, r -= a A p, s = D^-1 r, p = s + b p turn into
    scalar recurrences in an eigenvalue lam of D^-1 A:
        chi (x) starts at 1, sig (s) at -lam, pi (p) = sig (+ b pi), chi += a pi,
        sig -= a lam pi.
    (for b = 0 and x = x0 the first residual is s_0 = -D^-1 A x0 = -lam x0)."""
    lam = np.asarray(lam, dtype=np.float64)
    chi = np.ones_like(lam)
    sig = -lam.copy()
    pi = np.zeros_like(lam)
    for j, a in enumerate(alphas):
        pi = sig + (betas[j] * pi if j > 0 else 0.0)
        chi = chi + a * pi
        sig = sig - a * lam * pi
    return chi


def spectral_filter(G, x0, h, shift: float = 0.0):
    """h(D^-1 A) x0 with A = L + shift I, through the eigendecomposition of the symmetric
    M = D^-1/2 A D^-1/2 = V diag(mu) V^T:  D^-1/2 V diag(h(mu)) V^T D^1/2 x0."""
    A = G.dense("L") + shift * np.eye(G.n)
    ds = np.sqrt(G.d)
    M = A / ds[:, None] / ds[None, :]
    mu, V = np.linalg.eigh(0.5 * (M + M.T))
    return (V @ (h(mu) * (V.T @ (ds * x0)))) / ds, mu


def lowpass_projection(G, x0, k: int, pencil: str = "D"):
    """sum_{j<k} u_j u_j^T B x0 for the k lowest eigenvectors u_j of (L, B)."""
    lam, U = pencil_eig(G, pencil)
    b = G.d if pencil == "D" else np.ones(G.n)
    Uk = U[:, :k]
    return Uk @ (Uk.T @ (b * x0)), lam

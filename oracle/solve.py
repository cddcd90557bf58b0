"""Linear solves for the oracle.

Sec. 4.3: dynamic runs use implicit backward Euler with a conjugate gradient
solver.  ``pcg`` is textbook preconditioned CG with a block-Jacobi (3x3 node
block) preconditioner, stopping when ||r|| <= rtol ||b|| (the residual is
measured against the right-hand side, so a warm start cannot loosen the test).
``direct`` is a sparse LU solve (scipy), the exact solution up to rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def block_jacobi(A: sp.csr_matrix) -> np.ndarray:
    """Inverses of the 3x3 diagonal blocks of A, shape (n/3, 3, 3)."""
    n = A.shape[0] // 3
    D = np.zeros((n, 3, 3))
    Ad = A.tocsr()
    for a in range(3):
        for b in range(3):
            D[:, a, b] = Ad[np.arange(n) * 3 + a, np.arange(n) * 3 + b].A1
    return np.linalg.inv(D)


def pcg(A: sp.csr_matrix, b: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-6,
        maxit: int = 10000, Pinv: np.ndarray | None = None):
    """Preconditioned CG on the SPD system A x = b.

    Returns (x, iterations, ||b - A x|| / ||b||, status) with status 'ok',
    'maxiter' or 'breakdown' (p^T A p <= 0, e.g. an indefinite tangent).
    """
    if Pinv is None:
        Pinv = block_jacobi(A)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    r = b - A @ x
    if bnorm == 0.0 or np.linalg.norm(r) <= rtol * bnorm:
        return x, 0, (np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0), "ok"

    def prec(v):
        return np.einsum("nab,nb->na", Pinv, v.reshape(-1, 3)).ravel()

    z = prec(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        pq = p @ q
        if not pq > 0.0:
            return x, it, np.linalg.norm(r) / bnorm, "breakdown"
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        if rn <= rtol * bnorm:
            return x, it, rn / bnorm, "ok"
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(r) / bnorm, "maxiter"


def direct(A: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """Sparse LU solve (scipy SuperLU)."""
    return spla.spsolve(A.tocsc(), b)

"""The Chronopoulos-Gear form of projected block-Jacobi PCG (the quasi-static
inner solve's two-kernel loop) against the textbook three-step PCG of the
oracle, on small SPD block systems.

The recurrences are restated here in numpy in the kernels' order:
w = A z, gamma = r.z, delta = z.w (pinned rows of z and r are zero),
beta = gamma / gamma_old, p.A.p = delta - beta gamma / alpha_old,
alpha = gamma / p.A.p, then p = z + beta p, q = w + beta q, x += alpha p and
r -= alpha q on free rows, z = P r.  In exact arithmetic the iterates equal
textbook PCG's, so x after k iterations agrees to rounding and both stop after
the same number of iterations.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.solve import block_jacobi, pcg


def _spd_block_system(n_nodes, seed):
    rng = np.random.default_rng(seed)
    n = 3 * n_nodes
    # a sparse SPD matrix with 3x3 node blocks: a random graph Laplacian-like
    # coupling plus a diagonal shift
    rows, cols, vals = [], [], []
    for i in range(n_nodes):
        for j in rng.choice(n_nodes, size=4, replace=False):
            if j == i:
                continue
            B = rng.standard_normal((3, 3)) * 0.3
            for a in range(3):
                for b in range(3):
                    rows += [3 * i + a, 3 * j + a]
                    cols += [3 * j + b, 3 * i + b]
                    vals += [B[a, b], B[b, a]]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A = A + A.T
    shift = np.abs(A).sum(axis=1).A1 + rng.uniform(0.5, 2.0, n)
    A = (A + sp.diags(shift)).tocsr()
    return A, rng.standard_normal(n)


def _chronopoulos_gear(A, b, Pinv, free, k_max, rtol):
    """The two-kernel loop; rows with free == False are pinned (kept at x = 0)."""
    n = b.size
    fr = np.repeat(free, 3)

    def prec(v):
        return np.einsum("nab,nb->na", Pinv, v.reshape(-1, 3)).ravel()

    x = np.zeros(n)
    r = np.where(fr, b, 0.0)
    z = np.where(fr, prec(r), 0.0)
    bb = r @ r
    p = np.zeros(n)
    q = np.zeros(n)
    alpha = rz = 0.0
    k = 0
    while True:
        w = A @ z                      # k_qs_cg_spmv
        gamma, delta, rr = r @ z, z @ w, r @ r
        if rr <= rtol * rtol * bb or k >= k_max:
            return x, k
        beta = gamma / rz if k > 0 else 0.0
        den = delta - beta * gamma / alpha if k > 0 else delta
        assert den > 0.0
        alpha, rz = gamma / den, gamma
        if k == 0:                     # k_qs_cg_update
            p, q = z.copy(), w.copy()
        else:
            p, q = z + beta * p, w + beta * q
        x = np.where(fr, x + alpha * p, x)
        r = np.where(fr, r - alpha * q, 0.0)
        z = np.where(fr, prec(r), 0.0)
        k += 1


def _projected(A, free):
    """The free-free block of A (the projected system PCG solves), scattered back."""
    fr = np.repeat(free, 3)
    D = sp.diags(fr.astype(float))
    return (D @ A @ D + sp.diags((~fr).astype(float))).tocsr()


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("pinned", [False, True], ids=["free", "pinned"])
def test_chronopoulos_gear_iterates_match_textbook_pcg(seed, pinned):
    A, b = _spd_block_system(40, seed)
    free = np.ones(40, dtype=bool)
    if pinned:
        free[np.random.default_rng(seed + 10).choice(40, size=6, replace=False)] = False
    fr = np.repeat(free, 3)
    Ap = _projected(A, free)
    bp = np.where(fr, b, 0.0)
    Pinv = block_jacobi(A)
    for k in range(1, 12):
        x_ref, it, _, status = pcg(Ap, bp, rtol=1e-14, maxit=k, Pinv=Pinv)
        assert it == k and status == "maxiter"
        x_cg, kk = _chronopoulos_gear(A, b, Pinv, free, k, 1e-14)
        assert kk == k
        np.testing.assert_allclose(x_cg, x_ref, rtol=1e-9, atol=1e-12 * np.abs(x_ref).max())
        assert np.all(x_cg[~fr] == 0.0)


@pytest.mark.parametrize("seed", [3, 4])
def test_chronopoulos_gear_stops_with_textbook_pcg(seed):
    A, b = _spd_block_system(60, seed)
    free = np.ones(60, dtype=bool)
    Pinv = block_jacobi(A)
    x_ref, it_ref, rel, status = pcg(A, b, rtol=1e-6, maxit=1000, Pinv=Pinv)
    assert status == "ok"
    x_cg, it_cg = _chronopoulos_gear(A, b, Pinv, free, 1000, 1e-6)
    assert it_cg == it_ref
    np.testing.assert_allclose(x_cg, x_ref, rtol=1e-8, atol=1e-12 * np.abs(x_ref).max())

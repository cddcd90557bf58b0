"""The quasi-static nested solve (GF_QS_SOLVE_NESTED) restated in numpy: flexible
PCG in FP64 (Notay, 2000; one previous direction kept) whose preconditioner is
an inner PCG in FP32 on the matrix and block-Jacobi inverses rounded to FP32,
started from the outer residual scaled by 1 / |r_prev| and run until its
residual falls by the inner tolerance.

In the kernels' order, per outer iteration with z the inner solution, w = A z
and the previous direction p' (q' = A p'):
beta = z.q' / p'.q', p.q = z.w - 2 beta z.q' + beta^2 p'.q', alpha = p.r / p.q,
p = z - beta p', q = w - beta q', x += alpha p and r -= alpha q on free rows.

Pinned against what the mathematics fixes:
* the converged x solves the FP64 system (scipy's direct solve) to the outer
  tolerance, with pinned rows held at zero, on a stiff block system whose FP32
  rounding limits a single FP32 solve to a few digits;
* with an exact inner solve (FP64 direct solve as the preconditioner) the
  outer iteration stops after one step;
* the outer iterates do not depend on the inner scaling (FCG is invariant to a
  scalar multiple of the preconditioner's output), so the scaled and unscaled
  runs agree to rounding.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _stiff_block_system(n_nodes, seed, stiff=1e4):
    """A chain of 3x3 node blocks with a few random long-range couplings (SPD,
    condition number around 1e6-1e7: FP32 rounding of A then costs digits)."""
    rng = np.random.default_rng(seed)
    n = 3 * n_nodes
    rows, cols, vals = [], [], []

    def couple(i, j, B):
        for a in range(3):
            for b in range(3):
                rows.extend([3 * i + a, 3 * j + a, 3 * i + a, 3 * j + a])
                cols.extend([3 * j + b, 3 * i + b, 3 * i + b, 3 * j + b])
                vals.extend([-B[a, b], -B[b, a], B[a, b], B[a, b]])

    for i in range(n_nodes - 1):
        G = rng.standard_normal((3, 3)) * 0.1
        couple(i, i + 1, stiff * (np.eye(3) + 0.5 * (G + G.T)))
    for _ in range(n_nodes // 10):
        i, j = rng.choice(n_nodes, size=2, replace=False)
        couple(i, j, 1e-2 * stiff * np.eye(3))
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A = (A + A.T) * 0.5 + sp.eye(n) * 1e-3 * stiff
    return A.tocsr(), rng.standard_normal(n)


def _block_inverses(A, n_nodes):
    D = np.empty((n_nodes, 3, 3))
    Ad = A.tocsr()
    for i in range(n_nodes):
        D[i] = Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3].toarray()
    return np.linalg.inv(D)


def _inner_pcg32(A32, Pinv32, r, free, tol, maxit):
    """The inner two-kernel PCG in FP32 (dots in FP64), from r; returns d ~ A^-1 r."""
    fr = np.repeat(free, 3)

    def prec(v):
        return np.einsum("nab,nb->na", Pinv32, v.reshape(-1, 3)).ravel().astype(np.float32)

    r = np.where(fr, r, 0).astype(np.float32)
    z = np.where(fr, prec(r), 0).astype(np.float32)
    d = np.zeros_like(r)
    p = np.zeros_like(r)
    q = np.zeros_like(r)
    rr0 = float(np.dot(r.astype(np.float64), r))
    rz = float(np.dot(r.astype(np.float64), z))
    alpha = beta = 0.0
    k = 0
    while k < maxit:
        w = (A32 @ z).astype(np.float32)
        delta = float(np.dot(z.astype(np.float64), w))
        den = delta if k == 0 else delta - beta * rz / alpha
        if not den > 0:
            break
        alpha = rz / den
        p = z if k == 0 else (z + np.float32(beta) * p).astype(np.float32)
        q = w if k == 0 else (w + np.float32(beta) * q).astype(np.float32)
        d = np.where(fr, d + np.float32(alpha) * p, d).astype(np.float32)
        r = np.where(fr, r - np.float32(alpha) * q, 0).astype(np.float32)
        z = np.where(fr, prec(r), 0).astype(np.float32)
        rz_new = float(np.dot(r.astype(np.float64), z))
        rr = float(np.dot(r.astype(np.float64), r))
        k += 1
        beta = rz_new / rz
        rz = rz_new
        if rr <= tol * tol * rr0:
            break
    return d.astype(np.float64), k


def nested_solve(A, b, free, rtol, inner_tol=1e-2, scaled=True, inner=None, max_outer=500):
    """Flexible FP64 PCG around an inner solve; returns x, outer iterations, inner iterations."""
    n_nodes = b.size // 3
    fr = np.repeat(free, 3)
    A32 = A.astype(np.float32)
    Pinv32 = _block_inverses(A, n_nodes).astype(np.float32)
    x = np.zeros_like(b)
    r = np.where(fr, b, 0.0)
    bb = r @ r
    rr_prev = bb
    p = q = None
    pq = 0.0
    inner_total = 0
    for k in range(max_outer):
        if r @ r <= rtol * rtol * bb:
            return x, k, inner_total
        sc = 1.0 / np.sqrt(rr_prev) if scaled else 1.0
        if inner is None:
            z, its = _inner_pcg32(A32, Pinv32, sc * r, free, inner_tol, 10 * b.size)
        else:
            z, its = inner(sc * r), 1
        z = np.where(fr, z, 0.0)
        inner_total += its
        w = A @ z
        if k == 0:
            beta, pq_new, pr = 0.0, z @ w, z @ r
        else:
            zq = z @ q
            beta = zq / pq
            pq_new = z @ w - 2 * beta * zq + beta * beta * pq
            pr = z @ r - beta * (p @ r)
        alpha = pr / pq_new
        p = z if k == 0 else z - beta * p
        q = w if k == 0 else w - beta * q
        pq = pq_new
        rr_prev = r @ r
        x = np.where(fr, x + alpha * p, x)
        r = np.where(fr, r - alpha * q, 0.0)
    raise AssertionError("nested solve did not converge")


def _free_mask(n_nodes, seed):
    free = np.ones(n_nodes, bool)
    free[np.random.default_rng(seed).choice(n_nodes, size=max(1, n_nodes // 20), replace=False)] = False
    return free


def test_nested_solve_reaches_the_fp64_solution():
    A, b = _stiff_block_system(600, seed=3)
    free = _free_mask(600, seed=4)
    fr = np.repeat(free, 3)
    Aff = A[fr][:, fr]
    x_ref = spla.spsolve(Aff.tocsc(), b[fr])
    # one FP32 solve of the rounded system is good to a few digits only
    z32, _ = _inner_pcg32(A.astype(np.float32), _block_inverses(A, 600).astype(np.float32),
                          np.where(fr, b, 0), free, 1e-7, 100000)
    err32 = np.linalg.norm(z32[fr] - x_ref) / np.linalg.norm(x_ref)
    assert err32 > 1e-6
    x, outer, inner_total = nested_solve(A, b, free, rtol=1e-12)
    assert outer >= 2 and inner_total > outer
    np.testing.assert_array_equal(x[~fr], 0.0)
    res = np.linalg.norm(b[fr] - Aff @ x[fr]) / np.linalg.norm(b[fr])
    assert res <= 1e-12
    assert np.linalg.norm(x[fr] - x_ref) / np.linalg.norm(x_ref) < 1e3 * err32 * 1e-6


def test_exact_inner_solve_converges_in_one_outer_step():
    A, b = _stiff_block_system(200, seed=5)
    free = _free_mask(200, seed=6)
    fr = np.repeat(free, 3)
    lu = spla.splu(A[fr][:, fr].tocsc())

    def exact(v):
        out = np.zeros_like(v)
        out[fr] = lu.solve(v[fr])
        return out

    _, outer, _ = nested_solve(A, b, free, rtol=1e-10, inner=exact)
    assert outer == 1


def test_outer_iterates_do_not_depend_on_the_inner_scaling():
    A, b = _stiff_block_system(300, seed=7)
    free = _free_mask(300, seed=8)
    fr = np.repeat(free, 3)
    lu = spla.splu(A[fr][:, fr].tocsc())
    Pinv = _block_inverses(A, 300)

    def approx(v):   # a fixed SPD inexact preconditioner: A^-1 + 0.2 (block Jacobi)
        out = 0.2 * np.einsum("nab,nb->na", Pinv, v.reshape(-1, 3)).ravel()
        out[fr] += lu.solve(v[fr])
        return np.where(fr, out, 0.0)

    xs, outer_s, _ = nested_solve(A, b, free, rtol=1e-11, inner=approx, scaled=True)
    xu, outer_u, _ = nested_solve(A, b, free, rtol=1e-11, inner=approx, scaled=False)
    assert outer_s == outer_u and 2 <= outer_s <= 30
    np.testing.assert_allclose(xs, xu, rtol=1e-9, atol=1e-12 * np.abs(xu).max())

"""Pins of the oracle network (no GPU): manual gradients against central
finite differences, the block-Jacobi start at initialisation, SPD
preconditioner blocks, and bfloat16 rounding."""
import numpy as np
import pytest

from oracle import gnn


def small_problem(seed=0, n=40):
    rng = np.random.default_rng(seed)
    # random symmetric graph: a ring plus chords
    adj = {i: set() for i in range(n)}
    for i in range(n):
        for j in ((i + 1) % n, (i + 7) % n):
            adj[i].add(j)
            adj[j].add(i)
    row_ptr = [0]
    col = []
    for i in range(n):
        col += sorted(adj[i])
        row_ptr.append(len(col))
    E = len(col)
    g = gnn.Graph(row_ptr, col, rng.normal(size=(E, gnn.EIN)))
    f = rng.normal(size=(n, gnn.NIN))
    A = rng.normal(size=(n, 3, 3))
    Dinv = A @ np.swapaxes(A, 1, 2) + 0.5 * np.eye(3)
    C = gnn.block_inverse_cholesky(Dinv)
    b = rng.normal(size=(n, 3))
    dv = rng.normal(size=(n, 3))
    free = rng.uniform(size=n) > 0.1
    s = 0.7
    return g, f, C, b, dv, free, s, Dinv


def test_gradients_match_finite_differences():
    g, f, C, b, dv, free, s, _ = small_problem()
    params = gnn.init_params(3)
    rng = np.random.default_rng(4)
    for k in params:                       # make every path active (decoder not zero)
        params[k] = params[k] + 0.05 * rng.normal(size=params[k].shape)
    params["Wd"] = 0.02 * rng.normal(size=params["Wd"].shape)
    loss, grads = gnn.loss_and_grad(params, g, f, C, b, dv, free, s)
    vec = gnn.flatten(params)
    gvec = gnn.flatten(grads)
    offs = np.cumsum([0] + [int(np.prod(v)) for v in gnn.param_shapes().values()])
    idx = np.concatenate([rng.choice(np.arange(offs[i], offs[i + 1]), size=min(6, offs[i + 1] - offs[i]),
                                     replace=False) for i in range(len(offs) - 1)])
    h = 1e-6
    for i in idx:
        vp, vm = vec.copy(), vec.copy()
        vp[i] += h
        vm[i] -= h
        lp, _ = gnn.loss_and_grad(gnn.unflatten(vp), g, f, C, b, dv, free, s)
        lm, _ = gnn.loss_and_grad(gnn.unflatten(vm), g, f, C, b, dv, free, s)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gvec[i]) <= 1e-6 * max(abs(fd), 1e-2 * abs(loss)), (i, fd, gvec[i])


def test_initial_network_is_scaled_block_jacobi():
    g, f, C, b, dv, free, s, Dinv = small_problem(seed=1)
    out = gnn.forward(gnn.init_params(5), g, f)
    assert np.abs(out).max() == 0.0
    P, x0, _, _ = gnn.apply_outputs(out, C, b, s)
    np.testing.assert_allclose(P, (1 + gnn.EPS) * Dinv, rtol=1e-12)
    np.testing.assert_allclose(x0, (1 + gnn.EPS) * np.einsum("nab,nb->na", Dinv, b), rtol=1e-12)


def test_preconditioner_blocks_are_spd():
    g, f, C, b, dv, free, s, _ = small_problem(seed=2)
    params = gnn.init_params(6)
    params["Wd"] = 0.05 * np.random.default_rng(7).normal(size=params["Wd"].shape)
    P, _, _, _ = gnn.apply_outputs(gnn.forward(params, g, f), C, b, s)
    np.testing.assert_allclose(P, np.swapaxes(P, 1, 2), rtol=1e-12, atol=1e-14)
    assert np.linalg.eigvalsh(P).min() > 0


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e38, 1.0 + 2 ** -7])
    # bf16 keeps 8 significand bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    np.testing.assert_array_equal(gnn.to_bf16(vals)[[0, 1, 2, 3, 5]], [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0 + 2 ** -7])
    assert gnn.n_params() == sum(int(np.prod(s)) for s in gnn.param_shapes().values())

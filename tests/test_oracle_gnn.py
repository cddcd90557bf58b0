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
    R = rng.normal(size=(3 * n, 3 * n))
    Asys = R @ R.T / (3 * n) + np.eye(3 * n)              # SPD system
    return g, f, C, b, dv, free, s, Dinv, Asys


def test_gradients_match_finite_differences():
    g, f, C, b, dv, free, s, _, Asys = small_problem()
    params = gnn.init_params(3)
    rng = np.random.default_rng(4)
    for k in params:                       # make every path active (decoder not zero)
        params[k] = params[k] + 0.05 * rng.normal(size=params[k].shape)
    params["Wd"] = 0.02 * rng.normal(size=params["Wd"].shape)
    loss, grads = gnn.loss_and_grad(params, g, f, C, b, dv, free, s, Asys)
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
        lp, _ = gnn.loss_and_grad(gnn.unflatten(vp), g, f, C, b, dv, free, s, Asys)
        lm, _ = gnn.loss_and_grad(gnn.unflatten(vm), g, f, C, b, dv, free, s, Asys)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gvec[i]) <= 1e-6 * max(abs(fd), 1e-2 * abs(loss)), (i, fd, gvec[i])


def test_initial_network_is_scaled_block_jacobi():
    g, f, C, b, dv, free, s, Dinv, _ = small_problem(seed=1)
    out = gnn.forward(gnn.init_params(5), g, f)
    assert np.abs(out).max() == 0.0
    P, x0, _, _ = gnn.apply_outputs(out, C, b, s)
    np.testing.assert_allclose(P, (1 + gnn.EPS) * Dinv, rtol=1e-12)
    np.testing.assert_allclose(x0, (1 + gnn.EPS) * np.einsum("nab,nb->na", Dinv, b), rtol=1e-12)


def test_preconditioner_blocks_are_spd():
    g, f, C, b, dv, free, s, _, _ = small_problem(seed=2)
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


def test_build_inputs_hand_worked_three_nodes():
    """Network inputs of a 3-node path graph 0-1-2 worked by hand: node 2
    pinned, rest edge lengths 1 and 2 (mean 1.5), diagonal blocks with traces
    2, 4, 8 and known inverses."""
    import scipy.sparse as sp
    X = np.array([[0.0, 0, 0], [1, 0, 0], [1, 2, 0]])
    D = [2 * np.eye(3), np.array([[4.0, 1, 0], [1, 4, 0], [0, 0, 4]]), 8 * np.eye(3)]
    A01 = -0.5 * np.eye(3)
    A12 = np.zeros((3, 3))
    A12[0, 1] = 1.0
    A = np.zeros((9, 9))
    for i in range(3):
        A[3 * i:3 * i + 3, 3 * i:3 * i + 3] = D[i]
    A[0:3, 3:6], A[3:6, 0:3] = A01, A01.T
    A[3:6, 6:9], A[6:9, 3:6] = A12, A12.T
    b = np.array([[2.0, 0, 0], [5, 5, 0], [9, 9, 9]])
    mass = np.array([1.0, 2.0, 3.0])
    pinned = np.array([False, False, True])
    g, f, C, s, free, Dinv = gnn.build_inputs(sp.csr_matrix(A), mass, X, np.array([[0, 1], [1, 2]]), pinned, b)
    # y0 = [1, 0, 0], y1 = [1, 1, 0] (D1 [1, 1, 0] = [5, 5, 0]), y2 = 0 (pinned): s = sqrt(3 / 2)
    assert s == pytest.approx(np.sqrt(1.5), rel=1e-15)
    want = np.zeros((3, 16))
    want[:, 0] = np.log(np.array([2.0, 4.0, 8.0]) / (14.0 / 3.0))
    want[1, 4] = 0.25                                  # xy of D1 / 4 - I
    want[:, 7] = np.log(mass / 2.0)
    want[:, 8] = [0, 0, 1]
    want[:, 9] = np.array([1, 2, 1]) / 16.0
    want[0, 10:13] = np.array([1, 0, 0]) / np.sqrt(1.5)
    want[1, 10:13] = np.array([1, 1, 0]) / np.sqrt(1.5)
    np.testing.assert_allclose(f, want, rtol=1e-14, atol=1e-15)
    # rows: 0 <- 1 | 1 <- 0, 1 <- 2 | 2 <- 1
    assert list(g.row_ptr) == [0, 1, 3, 4] and list(g.col) == [1, 0, 2, 1]
    ew = np.zeros((4, 16))
    ew[0, 0:3], ew[0, 3:12] = [2 / 3, 0, 0], (A01 / np.sqrt(8)).ravel()
    ew[1, 0:3], ew[1, 3:12] = [-2 / 3, 0, 0], (A01.T / np.sqrt(8)).ravel()
    ew[2, 0:3], ew[2, 3:12] = [0, 4 / 3, 0], (A12 / np.sqrt(32)).ravel()
    ew[3, 0:3], ew[3, 3:12] = [0, -4 / 3, 0], (A12.T / np.sqrt(32)).ravel()
    np.testing.assert_allclose(g.efeat, ew, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(C[0], np.sqrt(0.5) * np.eye(3), rtol=1e-14)
    for i in range(3):
        np.testing.assert_allclose(C[i] @ C[i].T, np.linalg.inv(D[i]), rtol=1e-13, atol=1e-15)
        assert np.allclose(np.triu(C[i], 1), 0)
    assert list(free) == [True, True, False]


def test_energy_loss_of_a_scaled_target():
    """With target = c x0 the energy-norm loss is (1 - c)^2 / c^2 whatever A is,
    and the loss and every gradient vanish at target = x0."""
    g, f, C, b, dv, free, s, _, Asys = small_problem(seed=3)
    params = gnn.init_params(8)
    rng = np.random.default_rng(9)
    params["Wd"] = 0.05 * rng.normal(size=params["Wd"].shape)
    _, x0, _, _ = gnn.apply_outputs(gnn.forward(params, g, f), C, b, s)
    for c in (0.5, 2.0, -1.0):
        loss, _ = gnn.loss_and_grad(params, g, f, C, b, c * x0, free, s, Asys)
        assert loss == pytest.approx((1 - c) ** 2 / c ** 2, rel=1e-12)
    loss, grads = gnn.loss_and_grad(params, g, f, C, b, x0, free, s, Asys)
    assert loss == 0.0
    assert max(np.abs(v).max() for v in grads.values()) == 0.0


def test_training_pair_targets_solve_the_shifted_system():
    """training_pair: for dv solving the free system (pinned values prescribed),
    A_ff target = b_net on free rows, and target = 0, b_net = 0 on pinned ones."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    *_, Asys = small_problem(seed=4, n=30)
    n = 30
    rng = np.random.default_rng(5)
    pin = rng.uniform(size=n) < 0.2
    b = rng.normal(size=(n, 3))
    dv = np.zeros((n, 3))
    dv[pin] = rng.normal(size=(pin.sum(), 3))
    fr = np.repeat(~pin, 3)
    A = sp.csr_matrix(Asys)
    rhs = b.ravel()[fr] - A[fr][:, ~fr] @ dv.ravel()[~fr]
    dv.reshape(-1)[fr] = spl.spsolve(A[fr][:, fr].tocsc(), rhs)
    x_prev = rng.normal(size=(n, 3))
    bn, tg = gnn.training_pair(A, b, dv, x_prev, pin)
    np.testing.assert_allclose((A[fr][:, fr] @ tg.ravel()[fr]), bn.ravel()[fr], rtol=1e-10, atol=1e-12)
    assert np.abs(tg[pin]).max() == 0.0 and np.abs(bn[pin]).max() == 0.0

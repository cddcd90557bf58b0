"""Pins of the oracle's time step (no GPU): a one-tet step against a dense solve
with a finite-difference tangent, rest-state stationarity, CG against the
direct solve, and the plain-FEM limit of an unbroken mesh (chi = 1)."""
import numpy as np
import pytest

from oracle import elastic, solve
from oracle.step import Material, Model
from workloads import beam_config, single_tet


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.5, 2e-3)])
def test_single_tet_step_matches_dense_textbook_solve(alpha, beta):
    """Three nodes pinned, one free: one linearised backward-Euler step of
    M dv/dt = f(x, v), f = f_el(x) + f_ext - B v with Rayleigh B = alpha M + beta K
    (Sec. 3.1), written from the generic implicit update
    (M - dt df/dv - dt^2 df/dx) dv = dt (f + dt df/dx v),
    with df/dx = -K from finite differences of the Eq. 12 forces and a dense solve."""
    X, tets = single_tet()
    E, nu, rho, dt = 1e5, 0.3, 1000.0, 1e-2
    m = Model(X, tets, Material(E, nu, rho, threshold=np.inf, alpha=alpha, beta=beta))
    st = m.rest_state()
    st.x = X + np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0], [0.05, -0.03, 0.1]])
    st.v = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0], [0.2, 0.1, -0.3]])
    f_ext = np.zeros((4, 3))
    f_ext[3] = [1.0, 2.0, -3.0]
    new, info = m.step(st, dt, f_ext, pinned=np.array([0, 1, 2]))
    lam, mu = elastic.lame(E, nu)

    def force(xx):
        return elastic.element_forces(xx, tets, m.V, m.D2, m.q, lam, mu)[0, 3]

    h = 1e-7
    K = np.zeros((3, 3))
    for c in range(3):
        xp, xm = st.x.copy(), st.x.copy()
        xp[3, c] += h
        xm[3, c] -= h
        K[:, c] = -(force(xp) - force(xm)) / (2 * h)
    mass = rho * m.V[0] / 4
    B = alpha * mass * np.eye(3) + beta * K
    dfdx, dfdv = -K, -B
    f_total = force(st.x) + f_ext[3] - B @ st.v[3]
    A = mass * np.eye(3) - dt * dfdv - dt * dt * dfdx
    b = dt * (f_total + dt * dfdx @ st.v[3])
    dv = np.linalg.solve(A, b)
    np.testing.assert_allclose(new.v[3], st.v[3] + dv, rtol=1e-7)
    np.testing.assert_allclose(new.x[3], st.x[3] + dt * (st.v[3] + dv), rtol=1e-9)
    np.testing.assert_array_equal(new.v[:3], 0.0)


def test_rest_stays_at_rest():
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, threshold=np.inf, radius=w.radius))
    st = m.rest_state()
    new, info = m.step(st, w.dt, np.zeros_like(w.nodes), w.pinned)
    assert np.abs(new.v).max() < 1e-12
    assert np.abs(new.x - w.nodes).max() < 1e-14


def test_pcg_matches_direct_on_beam():
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, threshold=np.inf, radius=w.radius))
    st = m.rest_state()
    rng = np.random.default_rng(3)
    st.x = w.nodes + 0.01 * rng.normal(size=w.nodes.shape)
    st.v = 0.1 * rng.normal(size=w.nodes.shape)
    a, ia = m.step(st, w.dt, w.f_ext, w.pinned, solver="direct")
    b, ib = m.step(st, w.dt, w.f_ext, w.pinned, solver="pcg", rtol=1e-13)
    assert ib["status"] == "ok" and ib["iters"] > 0
    assert np.linalg.norm(a.v - b.v) <= 1e-10 * np.linalg.norm(a.v)


def test_unbroken_mesh_is_plain_fem():
    """Eq. 32-34 with chi = 1: the assembled K* and f* equal the plain sums of the
    F-route element forces (classical FEM) and their FD tangent is K*."""
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, threshold=np.inf, radius=0.0))
    rng = np.random.default_rng(4)
    x = w.nodes + 0.02 * rng.normal(size=w.nodes.shape)
    K, f = m.assemble(x, np.ones(len(w.tets)))
    assert abs(K - K.T).max() <= 1e-12 * abs(K).max()
    # net internal force vanishes (Newton's third law per element)
    assert np.abs(f.reshape(-1, 3).sum(0)).max() <= 1e-9 * np.abs(f).max()
    # directional FD of the assembled force along a random direction
    d = rng.normal(size=x.shape)
    h = 1e-7
    _, fp = m.assemble(x + h * d, np.ones(len(w.tets)))
    _, fm = m.assemble(x - h * d, np.ones(len(w.tets)))
    np.testing.assert_allclose(-(fp - fm) / (2 * h), K @ d.ravel(), rtol=1e-5, atol=1e-6 * np.abs(K @ d.ravel()).max())


def test_pcg_reports_breakdown_on_indefinite():
    import scipy.sparse as sp
    A = sp.csr_matrix(np.diag([1.0, 1.0, 1.0, -1.0, 1.0, 1.0]))
    b = np.ones(6)
    _, _, _, status = solve.pcg(A, b, rtol=1e-12, Pinv=np.tile(np.eye(3), (2, 1, 1)))
    assert status == "breakdown"


def test_prescribed_pinned_velocity():
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, threshold=np.inf, radius=0.0))
    st = m.rest_state()
    pv = np.tile([0.0, 0.01, -0.02], (len(w.pinned), 1))
    new, info = m.step(st, w.dt, w.f_ext, w.pinned, pinned_vel=pv)
    np.testing.assert_array_equal(new.v[w.pinned], pv)
    assert info["rel_res"] < 1e-12

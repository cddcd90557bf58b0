"""Pins of the oracle's consistent mass (Eq. 5) and of its Newton iterations
on the backward-Euler residual (no GPU).

Consistent mass: the quadrature of Eq. 5 against the textbook closed form of
the linear tet, m_ab = rho V (1 + delta_ab) / 20, and its row sums against the
lumped masses; a rigid translation is kept and the total momentum changes by
exactly dt sum f_ext (the internal forces of Eq. 12 sum to zero per tet).
Newton: one iteration is the linearised step; more iterations drive the
residual of the nonlinear backward-Euler equations to rounding, quadratically
when the damping matrix does not depend on the state (beta = 0)."""
import numpy as np
import pytest

from oracle import mesh
from oracle.step import Material, Model
from workloads import beam_config, single_tet
from helpers import deformed_state


def test_consistent_mass_matches_closed_form_and_lumped_row_sums():
    w = beam_config()
    V, _, _ = mesh.rest_geometry(w.nodes, w.tets)
    me = mesh.consistent_mass_blocks(w.tets, w.density, V)
    closed = w.density * V[:, None, None] * (np.ones((4, 4)) + np.eye(4)) / 20.0
    np.testing.assert_allclose(me, closed, rtol=1e-14, atol=0)
    M = mesh.consistent_mass_matrix(w.nodes, w.tets, w.density, V)
    lumped = mesh.lumped_mass(w.nodes, w.tets, w.density, V)
    np.testing.assert_allclose(np.asarray(M.sum(1)).ravel(), np.repeat(lumped, 3), rtol=1e-13)
    assert abs(M.sum() / 3 - w.density * V.sum()) <= 1e-12 * w.density * V.sum()


@pytest.mark.parametrize("mass", ["lumped", "consistent"])
def test_rigid_translation_is_kept(mass):
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, mass=mass))
    st = m.rest_state()
    st.v[:] = [0.3, -0.2, 0.1]
    new, _ = m.step(st, w.dt, np.zeros_like(w.nodes))
    np.testing.assert_allclose(new.v, st.v, rtol=0, atol=1e-12)


@pytest.mark.parametrize("mass", ["lumped", "consistent"])
@pytest.mark.parametrize("newton", [1, 3])
def test_momentum_changes_by_the_external_impulse(mass, newton):
    """No pins, no damping: sum over nodes of (M v) grows by dt sum f_ext
    (internal forces cancel per tet), for any number of Newton iterations."""
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, mass=mass))
    st = deformed_state(w, seed=3)
    f = np.random.default_rng(4).normal(size=w.nodes.shape) * 10.0
    new, _ = m.step(st, w.dt, f, newton_iters=newton)
    p0 = (m.M @ st.v.ravel()).reshape(-1, 3).sum(0)
    p1 = (m.M @ new.v.ravel()).reshape(-1, 3).sum(0)
    scale = np.abs(m.M @ st.v.ravel()).sum() + w.dt * np.abs(f).sum()
    np.testing.assert_allclose(p1 - p0, w.dt * f.sum(0), rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("mass", ["lumped", "consistent"])
@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.3, 1e-3)])
def test_one_newton_iteration_is_the_linearised_step(mass, alpha, beta):
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, alpha=alpha, beta=beta, mass=mass))
    st = deformed_state(w, seed=5)
    a, _ = m.step(st, w.dt, w.f_ext, w.pinned)
    b, info = m.step_newton(st, w.dt, w.f_ext, w.pinned, None, 1)
    dv = np.abs(a.v - st.v).max()
    np.testing.assert_allclose(b.v, a.v, rtol=0, atol=1e-11 * dv)
    np.testing.assert_allclose(b.x, a.x, rtol=0, atol=1e-11 * dv * w.dt + 1e-15)


def test_newton_converges_quadratically_to_the_backward_euler_solution():
    """A soft single tet with one free node under a large load: the linearised
    step leaves a large residual; Newton removes it quadratically (beta = 0,
    so the Jacobian is exact)."""
    X, tets = single_tet()
    m = Model(X, tets, Material(1e4, 0.3, 100.0))
    st = m.rest_state()
    f = np.zeros((4, 3))
    f[3] = [40.0, -30.0, 60.0]
    new, info = m.step(st, 5e-2, f, pinned=np.array([0, 1, 2]), newton_iters=8)
    res = info["newton_res"]
    assert res[1] > 1e-2 * res[0]                   # the linearised step is far from the solution
    assert info["final_res"] <= 1e-11 * res[0]
    k = next(i for i in range(1, len(res) - 1) if res[i + 1] < 1e-3 * res[i])
    assert res[k + 1] <= 10.0 * res[k] ** 2 / res[0]  # quadratic decrease near the solution
    # the solution satisfies the backward-Euler equations directly
    r, _ = m.newton_residual(st.x, st.v, new.v.ravel(), info["chi"], 5e-2, f)
    assert np.linalg.norm(r[9:]) <= 1e-11 * res[0]


def test_newton_with_damping_and_pins_converges_on_the_beam():
    w = beam_config()
    m = Model(w.nodes, w.tets, Material(w.young, w.poisson, w.density, alpha=0.2, beta=2e-3, mass="consistent"))
    st = deformed_state(w, seed=6, amp=0.08)
    vp = np.tile([0.0, 0.1, 0.0], (len(w.pinned), 1))
    new, info = m.step(st, 1e-2, w.f_ext, w.pinned, pinned_vel=vp, newton_iters=6)
    res = info["newton_res"]
    assert info["final_res"] <= 1e-8 * res[0]
    np.testing.assert_array_equal(new.v[w.pinned], vp)

"""Pins of the oracle's quasi-static load step (Eq. 36 with Newton and a line
search, Sec. 4.3), no GPU.

* A rigid translation of every pinned node with no load moves the whole body
  rigidly (the equilibrium is exact).
* The first Newton direction from rest is the linear-elastic solution
  K0 u = f (Eq. 36 at the rest tangent); the converged nonlinear answer differs
  from it by O(u^2), so halving the load shrinks the gap about fourfold.
* At convergence the residual f* + f_ext on free DOFs is at rounding level
  and the total energy decreased at every accepted step.
* With both ends pinned and one end pulled, the stretch gives the expected
  sign of the reaction and a stationary total energy along random free
  directions (first-order optimality checked by finite differences).
"""
import numpy as np
import pytest

from oracle.step import Material, Model
from workloads import kuhn_box


def bar(nz=6, energy="stvk"):
    X, T, grid = kuhn_box(2, 2, nz)
    m = Model(X, T, Material(1e6, 0.3, 1000.0, energy=energy))
    lo = np.nonzero(grid[:, 2] == 0)[0]
    hi = np.nonzero(grid[:, 2] == nz)[0]
    return m, X, lo, hi


@pytest.mark.parametrize("energy", ["stvk", "snh"])
def test_rigid_translation_of_the_supports(energy):
    m, X, lo, hi = bar(energy=energy)
    pins = np.concatenate([lo, hi])
    t = np.array([0.03, -0.02, 0.05])
    st = m.rest_state()
    new, info = m.quasistatic_step(st, np.zeros_like(X), pins, X[pins] + t)
    np.testing.assert_allclose(new.x, X + t, rtol=0, atol=1e-9 * np.abs(t).max())


def test_first_direction_is_linear_elasticity_and_the_gap_is_quadratic():
    m, X, lo, hi = bar()
    f = np.zeros_like(X)
    f[hi, 0] = 20.0                      # lateral tip load, base clamped
    gaps = []
    for scale in (1.0, 0.5):
        st = m.rest_state()
        K, _ = m.assemble(X, np.ones(len(m.tets)))
        free = np.repeat(np.isin(np.arange(len(X)), lo, invert=True), 3)
        u_lin = np.zeros(3 * len(X))
        u_lin[free] = np.linalg.solve(K[free][:, free].toarray(), scale * f.ravel()[free])
        new, info = m.quasistatic_step(st, scale * f, lo, None)
        u = (new.x - X).ravel()
        gaps.append(np.linalg.norm(u - u_lin) / np.linalg.norm(u_lin) ** 2)
        assert min(info["newton_res"]) <= 1e-9 * info["newton_res"][0]
    assert 0.7 <= gaps[1] / gaps[0] <= 1.3      # |u - u_lin| ~ C |u|^2 with a load-independent C


@pytest.mark.parametrize("energy", ["stvk", "snh"])
def test_pulled_bar_reaches_equilibrium_with_decreasing_energy(energy):
    m, X, lo, hi = bar(energy=energy)
    pins = np.concatenate([lo, hi])
    target = X[pins].copy()
    target[len(lo):, 2] += 0.6            # stretch by 10%
    st = m.rest_state()
    new, info = m.quasistatic_step(st, np.zeros_like(X), pins, target)
    res = info["newton_res"]
    assert min(res) <= 1e-9 * res[0]
    e = info["energies"]
    assert all(b < a for a, b in zip(e, e[1:]))
    # stationarity: directional derivatives of E along random free directions vanish
    chi = np.ones(len(m.tets))
    rng = np.random.default_rng(0)
    E0 = m.total_energy(new.x, chi, np.zeros_like(X))
    scale = abs(E0) / np.abs(new.x - X).max()
    for _ in range(3):
        d = rng.normal(size=X.shape)
        d[pins] = 0.0
        h = 1e-5
        dE = (m.total_energy(new.x + h * d, chi, np.zeros_like(X)) -
              m.total_energy(new.x - h * d, chi, np.zeros_like(X))) / (2 * h)
        assert abs(dE) <= 1e-6 * scale * np.abs(d).max()
    # the pulled end feels a restoring force (reaction along -z on the moved face)
    K, f = m.assemble(new.x, chi)
    assert f.reshape(-1, 3)[hi, 2].sum() < 0

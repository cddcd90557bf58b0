"""Pins of the oracle's elastic part against the mathematics (no GPU).

Each check uses something other than the oracle's own formulas: the
deformation-gradient route of classical FEM (Table 1, Eq. 32), closed forms for
uniaxial stretch, finite differences, rigid-motion invariance, and symmetry.
"""
import numpy as np
import pytest

from oracle import elastic, mesh
from workloads import single_tet


def random_tets(n, seed=0):
    """Well-shaped random tets: a regular tet, perturbed by 15% of its edge,
    randomly rotated, scaled and translated (one tet per 4 fresh nodes)."""
    rng = np.random.default_rng(seed)
    reg = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(8)
    X = []
    for _ in range(n):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        P = (reg + 0.15 * rng.uniform(-1, 1, size=(4, 3))) @ R.T * rng.uniform(0.5, 2.0)
        X.append(P + rng.normal(size=3))
    X = np.concatenate(X)
    tets = np.arange(4 * n, dtype=np.int64).reshape(n, 4)
    return X, tets


def F_route(X, x, tets):
    """Deformation gradient F = Ds Dm^-1 (Table 1) per tet."""
    P, p = X[tets], x[tets]
    Dm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2)
    Ds = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], 2)
    return Ds @ np.linalg.inv(Dm), Dm


def test_C_from_edge_lengths_equals_FtF():
    """Thm 3.1: the Eq. 31 least-squares C equals F^T F for any non-degenerate tet."""
    X, tets = random_tets(200)
    rng = np.random.default_rng(1)
    x = X + 0.3 * rng.normal(size=X.shape)
    F, _ = F_route(X, x, tets)
    V, D2, q = mesh.rest_geometry(X, tets)
    C = elastic.cauchy_green_lsq(elastic.squared_edge_lengths(x, tets), D2, q)
    Cref = np.einsum("tki,tkj->tij", F, F)
    assert np.max(np.abs(C - Cref)) <= 1e-11 * np.max(np.abs(Cref))


@pytest.mark.parametrize("eps", [0.05, -0.02, 0.3])
def test_uniaxial_stretch_closed_form(eps):
    """Single tet, F = diag(1+eps,1,1): Eq. 37 in edge lengths equals
    V [mu E:E + lam/2 (tr E)^2] and I_C = (1+eps)^2+2, II_C = (1+eps)^4+2."""
    X, tets = single_tet()
    x = X.copy()
    x[:, 0] *= 1 + eps
    E, nu = 1e6, 0.3
    lam, mu = elastic.lame(E, nu)
    V, D2, q = mesh.rest_geometry(X, tets)
    s = elastic.squared_edge_lengths(x, tets)
    C = elastic.cauchy_green_lsq(s, D2, q)[0]
    assert np.trace(C) == pytest.approx((1 + eps) ** 2 + 2, rel=1e-13)
    assert np.sum(C * C) == pytest.approx((1 + eps) ** 4 + 2, rel=1e-13)
    Eg = np.diag([((1 + eps) ** 2 - 1) / 2, 0, 0])
    psi_F = (1 / 6) * (mu * np.sum(Eg * Eg) + lam / 2 * np.trace(Eg) ** 2)
    psi = elastic.element_energy(x, tets, V, D2, q, lam, mu)[0]
    assert psi == pytest.approx(psi_F, rel=1e-12)


def test_force_matches_F_route_and_balances():
    """Eq. 12 edge forces equal the classical -V P(F) dF/dx forces (Eq. 32) and
    sum to zero force and zero torque per element."""
    X, tets = random_tets(100, seed=3)
    rng = np.random.default_rng(4)
    x = X + 0.2 * rng.normal(size=X.shape)
    lam, mu = elastic.lame(5e5, 0.35)
    V, D2, q = mesh.rest_geometry(X, tets)
    f = elastic.element_forces(x, tets, V, D2, q, lam, mu)
    F, Dm = F_route(X, x, tets)
    Eg = 0.5 * (np.einsum("tki,tkj->tij", F, F) - np.eye(3))
    S = lam * np.trace(Eg, axis1=1, axis2=2)[:, None, None] * np.eye(3) + 2 * mu * Eg
    P = F @ S
    H = -V[:, None, None] * P @ np.linalg.inv(Dm).transpose(0, 2, 1)   # forces on nodes 1..3
    fref = np.concatenate([-H.sum(2)[:, None, :], H.transpose(0, 2, 1)], 1)
    scale = np.abs(fref).max()
    assert np.max(np.abs(f - fref)) <= 1e-10 * scale
    assert np.max(np.abs(f.sum(1))) <= 1e-10 * scale
    torque = np.cross(x[tets], f).sum(1)
    assert np.max(np.abs(torque)) <= 1e-9 * scale


def test_forces_and_tangent_by_finite_differences():
    """f = -d(V Psi)/dx and K = -df/dx by central differences (h = 1e-6)."""
    X, tets = random_tets(20, seed=5)
    rng = np.random.default_rng(6)
    x = X + 0.1 * rng.normal(size=X.shape)
    lam, mu = elastic.lame(1e6, 0.3)
    V, D2, q = mesh.rest_geometry(X, tets)
    f = elastic.element_forces(x, tets, V, D2, q, lam, mu)
    K = elastic.element_tangent(x, tets, V, D2, q, lam, mu)
    h = 1e-6
    for e in range(len(tets)):
        fd_f = np.zeros(12)
        fd_K = np.zeros((12, 12))
        for a in range(4):
            for c in range(3):
                xp, xm = x.copy(), x.copy()
                xp[tets[e, a], c] += h
                xm[tets[e, a], c] -= h
                Ep = elastic.element_energy(xp, tets[e:e + 1], V[e:e + 1], D2[e:e + 1], q[e:e + 1], lam, mu)[0]
                Em = elastic.element_energy(xm, tets[e:e + 1], V[e:e + 1], D2[e:e + 1], q[e:e + 1], lam, mu)[0]
                fd_f[3 * a + c] = -(Ep - Em) / (2 * h)
                fp = elastic.element_forces(xp, tets[e:e + 1], V[e:e + 1], D2[e:e + 1], q[e:e + 1], lam, mu)[0]
                fm = elastic.element_forces(xm, tets[e:e + 1], V[e:e + 1], D2[e:e + 1], q[e:e + 1], lam, mu)[0]
                fd_K[:, 3 * a + c] = -(fp - fm).ravel() / (2 * h)
        assert np.max(np.abs(fd_f - f[e].ravel())) <= 1e-7 * np.abs(f[e]).max()
        assert np.max(np.abs(fd_K - K[e])) <= 1e-7 * np.abs(K[e]).max()


def test_tangent_symmetric_and_rigid_modes_at_rest():
    """k_e is symmetric; at rest its null space holds the 6 rigid modes."""
    X, tets = random_tets(30, seed=7)
    lam, mu = elastic.lame(1e6, 0.3)
    V, D2, q = mesh.rest_geometry(X, tets)
    K = elastic.element_tangent(X, tets, V, D2, q, lam, mu)
    assert np.max(np.abs(K - K.transpose(0, 2, 1))) <= 1e-14 * np.abs(K).max() * 10
    P = X[tets]
    for e in range(len(tets)):
        modes = []
        for c in range(3):
            t = np.zeros((4, 3))
            t[:, c] = 1
            modes.append(t.ravel())
            w = np.zeros(3)
            w[c] = 1
            modes.append(np.cross(w, P[e] - P[e].mean(0)).ravel())
        R = np.stack(modes, 1)
        assert np.max(np.abs(K[e] @ R)) <= 1e-9 * np.abs(K[e]).max()
        ev = np.linalg.eigvalsh(K[e])
        assert np.sum(np.abs(ev) <= 1e-9 * np.abs(ev).max()) == 6


def test_rigid_motion_invariance():
    """x -> R x + t leaves V Psi unchanged and rotates the forces."""
    X, tets = random_tets(50, seed=8)
    rng = np.random.default_rng(9)
    x = X + 0.2 * rng.normal(size=X.shape)
    Rq, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Rq) < 0:
        Rq[:, 0] *= -1
    xr = x @ Rq.T + np.array([1.0, -2.0, 3.0])
    lam, mu = elastic.lame(1e6, 0.3)
    V, D2, q = mesh.rest_geometry(X, tets)
    e0 = elastic.element_energy(x, tets, V, D2, q, lam, mu)
    e1 = elastic.element_energy(xr, tets, V, D2, q, lam, mu)
    assert np.allclose(e0, e1, rtol=1e-11, atol=0)
    f0 = elastic.element_forces(x, tets, V, D2, q, lam, mu)
    f1 = elastic.element_forces(xr, tets, V, D2, q, lam, mu)
    assert np.max(np.abs(f0 @ Rq.T - f1)) <= 1e-10 * np.abs(f0).max()
    # rest state: no force, no energy
    f_rest = elastic.element_forces(X, tets, V, D2, q, lam, mu)
    assert np.max(np.abs(f_rest)) <= 1e-9 * lam


def test_edge_hessian_is_not_diagonal():
    """Sec. 5.5 (Eq. 38 contrast): the energy is not a sum of per-edge terms, so
    d2Psi/ds_k ds_l has non-zero off-diagonal entries."""
    X, tets = single_tet()
    lam, mu = elastic.lame(1e6, 0.3)
    V, D2, q = mesh.rest_geometry(X, tets)
    _, _, H, _ = elastic.edge_derivatives(X, tets, D2, q, lam, mu)
    off = H[0] - np.diag(np.diag(H[0]))
    assert np.abs(off).max() > 1e-3 * np.abs(np.diag(H[0])).max()

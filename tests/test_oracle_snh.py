"""Pins of the oracle's stable Neo-Hookean energy (Eq. 35, squared reading,
signed J) written in squared edge lengths (no GPU).

The oracle takes the paper's route: C from the edge lengths by Eq. 31, the
energy and its edge-space derivatives by the chain rule.  Here it is checked
against the deformation-gradient form written out independently in this file
(F = Ds Dm^-1, P = dPsi/dF = mu (1 - 1/(I_C + 1)) F + lam (J - a) cof F),
finite differences, rigid motions, the stress-free rest state, symmetry of the
tangent and the behaviour of an inverted tet."""
import numpy as np
import pytest

from oracle import damage, elastic, mesh
from workloads import beam_config

E, NU = 1e6, 0.3
LAM, MU = elastic.lame(E, NU)
A = 1.0 + MU / LAM - MU / (4.0 * LAM)


def random_tets(n=40, seed=0, amp=0.25):
    rng = np.random.default_rng(seed)
    X = np.zeros((4 * n, 3))
    tets = np.arange(4 * n).reshape(n, 4)
    for e in range(n):
        P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) + 0.1 * rng.normal(size=(4, 3))
        if np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1)) < 0:
            P[[1, 2]] = P[[2, 1]]
        X[4 * e:4 * e + 4] = P
    x = X + amp * rng.normal(size=X.shape) * 0.2
    return X, x, tets


def f_route(X, x, tets):
    """Psi, P and nodal forces from F directly (independent of the edge route)."""
    P0, P1 = X[tets], x[tets]
    Dm = np.stack([P0[:, 1] - P0[:, 0], P0[:, 2] - P0[:, 0], P0[:, 3] - P0[:, 0]], 2)
    Ds = np.stack([P1[:, 1] - P1[:, 0], P1[:, 2] - P1[:, 0], P1[:, 3] - P1[:, 0]], 2)
    B = np.linalg.inv(Dm)
    F = Ds @ B
    V = np.abs(np.linalg.det(Dm)) / 6.0
    IC = np.einsum("tij,tij->t", F, F)
    J = np.linalg.det(F)
    psi = MU / 2 * (IC - 3) + LAM / 2 * (J - A) ** 2 - MU / 2 * np.log(IC + 1)
    cof = J[:, None, None] * np.linalg.inv(F).transpose(0, 2, 1)
    Pk = (MU * (1 - 1 / (IC + 1)))[:, None, None] * F + (LAM * (J - A))[:, None, None] * cof
    G = np.concatenate([-B.sum(1, keepdims=True), B], 1)        # (t, 4, 3): dF_ij/dx_a,c = delta_ic G_aj
    f = -V[:, None, None] * np.einsum("tcj,taj->tac", Pk, G)
    return V * psi, Pk, f, J


def edge_route(X, x, tets):
    V, D2, q = mesh.rest_geometry(X, tets)
    psi = elastic.element_energy(x, tets, V, D2, q, LAM, MU, energy="snh")
    f = elastic.element_forces(x, tets, V, D2, q, LAM, MU, energy="snh")
    K = elastic.element_tangent(x, tets, V, D2, q, LAM, MU, energy="snh")
    return psi, f, K, (V, D2, q)


def test_edge_route_equals_deformation_gradient_route():
    X, x, tets = random_tets()
    psi_f, _, f_f, J = f_route(X, x, tets)
    psi_e, f_e, _, _ = edge_route(X, x, tets)
    assert (J > 0).all()
    np.testing.assert_allclose(psi_e, psi_f, rtol=1e-11, atol=1e-12 * np.abs(psi_f).max())
    np.testing.assert_allclose(f_e, f_f, rtol=1e-9, atol=1e-11 * np.abs(f_f).max())


def test_inverted_tet_uses_the_signed_J():
    """Move node 3 through the opposite face: J < 0, the edge lengths alone
    would give |J|.  Energy and forces still match the F route, and the force
    on the flipped node points back (a small step along it raises J)."""
    X, x, tets = random_tets(n=6, seed=3, amp=0.0)
    for e in range(len(tets)):
        p = x[tets[e]]
        n = np.cross(p[1] - p[0], p[2] - p[0])
        n /= np.linalg.norm(n)
        x[tets[e, 3]] = p[3] - 1.4 * np.dot(p[3] - p[0], n) * n
    psi_f, _, f_f, J = f_route(X, x, tets)
    psi_e, f_e, _, _ = edge_route(X, x, tets)
    assert (J < 0).all()
    np.testing.assert_allclose(psi_e, psi_f, rtol=1e-11)
    np.testing.assert_allclose(f_e, f_f, rtol=1e-9, atol=1e-11 * np.abs(f_f).max())
    x2 = x.copy()
    x2[tets[:, 3]] += 1e-4 * f_e[:, 3] / np.abs(f_e[:, 3]).max()
    assert (f_route(X, x2, tets)[3] > J).all()


def test_rest_state_is_stress_free():
    w = beam_config()
    V, D2, q = mesh.rest_geometry(w.nodes, w.tets)
    f = elastic.element_forces(w.nodes, w.tets, V, D2, q, LAM, MU, energy="snh")
    assert np.abs(f).max() <= 1e-9 * MU
    C = np.broadcast_to(np.eye(3), (3, 3, 3)).copy()
    S = damage.stress_voigt(C, LAM, MU, "snh", np.ones(3))
    assert np.abs(S).max() <= 1e-9 * MU


def test_forces_and_tangent_against_finite_differences():
    X, x, tets = random_tets(n=3, seed=5)
    psi, f, K, (V, D2, q) = edge_route(X, x, tets)
    h = 1e-6
    for e in range(len(tets)):
        te = tets[e:e + 1]
        args = (V[e:e + 1], D2[e:e + 1], q[e:e + 1], LAM, MU)
        for a in range(4):
            for c in range(3):
                xp, xm = x.copy(), x.copy()
                xp[te[0, a], c] += h
                xm[te[0, a], c] -= h
                ep = elastic.element_energy(xp, te, *args, energy="snh")[0]
                em = elastic.element_energy(xm, te, *args, energy="snh")[0]
                assert abs(-(ep - em) / (2 * h) - f[e, a, c]) <= 1e-6 * np.abs(f[e]).max()
                fp = elastic.element_forces(xp, te, *args, energy="snh")[0]
                fm = elastic.element_forces(xm, te, *args, energy="snh")[0]
                col = -(fp - fm).ravel() / (2 * h)
                np.testing.assert_allclose(K[e][:, 3 * a + c], col, rtol=0, atol=1e-6 * np.abs(K[e]).max())
    np.testing.assert_allclose(K, K.transpose(0, 2, 1), rtol=0, atol=1e-12 * np.abs(K).max())


def test_rigid_motion_invariance():
    X, x, tets = random_tets(n=10, seed=7)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    xr = x @ R.T + np.array([3.0, -1.0, 2.0])
    p0, f0, _, _ = edge_route(X, x, tets)
    p1, f1, _, _ = edge_route(X, xr, tets)
    np.testing.assert_allclose(p1, p0, rtol=1e-10)
    np.testing.assert_allclose(f1, f0 @ R.T, rtol=0, atol=1e-9 * np.abs(f0).max())


def test_second_pk_stress_matches_the_f_route():
    """P = F S with S = 2 dPsi/dC of the damage criterion (Eq. 14)."""
    X, x, tets = random_tets(n=12, seed=9)
    _, Pk, _, J = f_route(X, x, tets)
    V, D2, q = mesh.rest_geometry(X, tets)
    s = elastic.squared_edge_lengths(x, tets)
    C = elastic.cauchy_green_lsq(s, D2, q)
    Sv = damage.stress_voigt(C, LAM, MU, "snh", J)
    S = np.zeros((len(tets), 3, 3))
    for k, (i, j) in enumerate(damage.VOIGT):
        S[:, i, j] = S[:, j, i] = Sv[:, k]
    P0, P1 = X[tets], x[tets]
    Dm = np.stack([P0[:, 1] - P0[:, 0], P0[:, 2] - P0[:, 0], P0[:, 3] - P0[:, 0]], 2)
    Ds = np.stack([P1[:, 1] - P1[:, 0], P1[:, 2] - P1[:, 0], P1[:, 3] - P1[:, 0]], 2)
    F = Ds @ np.linalg.inv(Dm)
    np.testing.assert_allclose(F @ S, Pk, rtol=0, atol=1e-9 * np.abs(Pk).max())


@pytest.mark.parametrize("eps", [0.05, -0.1])
def test_uniaxial_stretch_closed_form(eps):
    """F = diag(1 + eps, 1, 1): I_C = (1 + eps)^2 + 2, J = 1 + eps."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    x = X.copy()
    x[:, 0] *= 1 + eps
    V, D2, q = mesh.rest_geometry(X, np.arange(4)[None])
    psi = elastic.element_energy(x, np.arange(4)[None], V, D2, q, LAM, MU, energy="snh")[0]
    IC = (1 + eps) ** 2 + 2
    want = V[0] * (MU / 2 * (IC - 3) + LAM / 2 * (1 + eps - A) ** 2 - MU / 2 * np.log(IC + 1))
    assert abs(psi - want) <= 1e-12 * abs(want)

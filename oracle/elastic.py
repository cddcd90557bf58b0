"""Hyperelastic element quantities written in squared edge lengths (oracle).

Paper passages followed:
* Eq. 27: lambda_mn^2 = (d_mn / D_mn)^2, the squared stretch of each edge.
* Eq. 28-31 (Thm 3.1): C solves  min ||C . Q - Lambda||^2  with Q_mn = q_mn (x) q_mn
  built from the unit edge direction; the closed form is
  C = Lambda . [Q (x) Q]^+ . Q  (^+ = pseudo-inverse).  Reading used: q_mn is the
  REST unit edge, so that C . Q_mn = lambda_mn^2 holds exactly for C = F^T F.
* Eq. 37: Saint-Venant-Kirchhoff  Psi = lam/8 (I_C-3)^2 + mu/4 (II_C - 2 I_C + 3).
* Eq. 35: stable Neo-Hookean  Psi = mu/2 (I_C - 3) + lam/2 (J - a)^2 - mu/2 log(I_C + 1),
  a = 1 + mu/lam - mu/(4 lam).  Reading used: the (J - a) term is squared (as
  in the energy the paper cites for it; printed without the square, the rest
  state would carry a stress lam/2), and J is the signed det F: its magnitude
  sqrt(det C) is a function of the edge lengths, its sign the orientation of
  the current tet relative to the rest tet.
* Eq. 12: f_i = -V dPsi/dr_i = 2V sum_j dPsi/d(d_ij^2) d_ij dhat_ij, with dhat_ij
  the unit vector from node i to node j (the restoring sign).
* Eq. 10/11 and Eq. 33: the tangent k_e is the Hessian of the element energy;
  Eq. 32-34: f* = chi f, k* = chi k with chi frozen.

All arrays are batched over tets; float64 throughout.
"""
from __future__ import annotations

import numpy as np

from .mesh import LOCAL_EDGES


def lame(young: float, poisson: float):
    """Lame parameters (lam, mu) of an isotropic material."""
    lam = young * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson))
    mu = young / (2.0 * (1.0 + poisson))
    return lam, mu


def squared_edge_lengths(x: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """s_k = (d_mn)^2 for the 6 local edges of Eq. 15, current positions."""
    P = x[np.asarray(tets, np.int64)]
    ev = np.stack([P[:, b] - P[:, a] for a, b in LOCAL_EDGES], 1)
    return np.einsum("tki,tki->tk", ev, ev)


def _Q(q: np.ndarray) -> np.ndarray:
    """Q_mn = q_mn (x) q_mn (Eq. 28), shape (t, 6, 3, 3)."""
    return q[..., :, None] * q[..., None, :]


def lsq_operator(D2: np.ndarray, q: np.ndarray) -> np.ndarray:
    """dC/ds_k for each tet: the (t, 6, 3, 3) tensors M_k such that the Eq. 31
    solution is C = sum_k s_k M_k.  With Lambda_k = s_k / D_k^2 (Eq. 27) and
    C = Lambda . [Q (x) Q]^+ . Q (Eq. 31):  M_k = (1/D_k^2) sum_l [QQ^+]_kl Q_l."""
    Q = _Q(q)
    QQ = np.einsum("tkij,tlij->tkl", Q, Q)          # [Q (x) Q]_kl = Q_k : Q_l
    QQp = np.linalg.pinv(QQ)                         # pseudo-inverse of Eq. 31
    return np.einsum("tkl,tlij->tkij", QQp, Q) / D2[:, :, None, None]


def cauchy_green_lsq(s: np.ndarray, D2: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Right Cauchy-Green tensor from squared edge lengths (Eq. 27-31).

    Lambda (Eq. 27/29) -> C = Lambda . [Q (x) Q]^+ . Q (Eq. 31)."""
    Q = _Q(q)
    Lam = s / D2                                      # Eq. 27
    QQ = np.einsum("tkij,tlij->tkl", Q, Q)
    QQp = np.linalg.pinv(QQ)
    return np.einsum("tk,tkl,tlij->tij", Lam, QQp, Q)


def stvk_density(C: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """Eq. 37 with I_C = tr C and II_C = C : C (Table 1)."""
    I = np.trace(C, axis1=-2, axis2=-1)
    II = np.einsum("...ij,...ij->...", C, C)
    return lam / 8.0 * (I - 3.0) ** 2 + mu / 4.0 * (II - 2.0 * I + 3.0)


def stvk_dpsi_dC(C: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """dPsi/dC of Eq. 37: lam/4 (I_C - 3) Id + mu/2 (C - Id)."""
    I = np.trace(C, axis1=-2, axis2=-1)
    eye = np.eye(3)
    return lam / 4.0 * (I - 3.0)[..., None, None] * eye + mu / 2.0 * (C - eye)


def stvk_d2psi_dC2(A: np.ndarray, B: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """Second derivative of Eq. 37 applied to two symmetric directions:
    d2Psi/dC2 [A, B] = lam/4 tr A tr B + mu/2 A : B (constant in C)."""
    trA = np.trace(A, axis1=-2, axis2=-1)
    trB = np.trace(B, axis1=-2, axis2=-1)
    return lam / 4.0 * trA * trB + mu / 2.0 * np.einsum("...ij,...ij->...", A, B)


def snh_alpha(lam: float, mu: float) -> float:
    """a of Eq. 35 (the rest state F = I is stress-free with the squared term)."""
    return 1.0 + mu / lam - mu / (4.0 * lam)


def orientation(x: np.ndarray, tets: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Sign of det F per tet: sign(det Ds) sign(det Dm), with the rest sign read
    from the rest unit edges q of local edges (0,1) (0,2) (0,3)."""
    P = x[np.asarray(tets, np.int64)]
    Ds = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2)
    Qm = np.stack([q[:, 0], q[:, 1], q[:, 2]], 2)
    return np.sign(np.linalg.det(Ds)) * np.sign(np.linalg.det(Qm))


def snh_density(IC, J, lam: float, mu: float):
    """Eq. 35 (squared reading) from I_C = tr C and the signed J."""
    a = snh_alpha(lam, mu)
    return mu / 2.0 * (IC - 3.0) + lam / 2.0 * (J - a) ** 2 - mu / 2.0 * np.log(IC + 1.0)


def edge_derivatives(x: np.ndarray, tets: np.ndarray, D2: np.ndarray, q: np.ndarray,
                     lam: float, mu: float, energy: str = "stvk"):
    """g_k = dPsi/ds_k (t, 6) and H_kl = d2Psi/ds_k ds_l (t, 6, 6) by the chain
    rule through the linear map s -> C = sum_k s_k M_k of Eq. 31.  Also returns
    Psi and C.

    energy "stvk" (Eq. 37): g = dPsi/dC : M_k, H = d2Psi/dC2 [M_k, M_l].
    energy "snh" (Eq. 35): with I_C = sum_k s_k tr M_k, J = sgn sqrt(det C),
    dJ/ds_k = J/2 tr(C^-1 M_k) and d2J/ds_k ds_l = J/4 t_k t_l - J/2 tr(C^-1 M_l C^-1 M_k)
    (t_k = tr(C^-1 M_k)), from d det C = det C tr(C^-1 dC)."""
    s = squared_edge_lengths(x, tets)
    M = lsq_operator(D2, q)
    C = np.einsum("tk,tkij->tij", s, M)
    if energy == "stvk":
        dPdC = stvk_dpsi_dC(C, lam, mu)
        g = np.einsum("tij,tkij->tk", dPdC, M)
        H = stvk_d2psi_dC2(M[:, :, None], M[:, None, :], lam, mu)
        return stvk_density(C, lam, mu), g, H, C
    if energy != "snh":
        raise ValueError(f"unknown energy {energy!r}")
    a = snh_alpha(lam, mu)
    IC = np.trace(C, axis1=-2, axis2=-1)
    J = orientation(x, tets, q) * np.sqrt(np.linalg.det(C))
    trM = np.trace(M, axis1=-2, axis2=-1)                       # (t, 6)
    Ci = np.linalg.inv(C)
    CiM = np.einsum("tij,tkjl->tkil", Ci, M)                    # C^-1 M_k
    t = np.trace(CiM, axis1=-2, axis2=-1)
    Jk = 0.5 * J[:, None] * t
    Jkl = 0.25 * J[:, None, None] * t[:, :, None] * t[:, None, :] \
        - 0.5 * J[:, None, None] * np.einsum("tkij,tlji->tkl", CiM, CiM)
    w = 1.0 / (IC + 1.0)
    g = mu / 2.0 * trM * (1.0 - w)[:, None] + lam * (J - a)[:, None] * Jk
    H = mu / 2.0 * (w * w)[:, None, None] * trM[:, :, None] * trM[:, None, :] \
        + lam * (Jk[:, :, None] * Jk[:, None, :] + (J - a)[:, None, None] * Jkl)
    return snh_density(IC, J, lam, mu), g, H, C


def grad_s(x: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """ds_k/dx over the 12 element DOFs (node-major: node a -> 3a..3a+2), (t, 6, 12)."""
    P = x[np.asarray(tets, np.int64)]
    out = np.zeros((P.shape[0], 6, 12))
    for k, (a, b) in enumerate(LOCAL_EDGES):
        d = P[:, b] - P[:, a]
        out[:, k, 3 * a:3 * a + 3] = -2.0 * d
        out[:, k, 3 * b:3 * b + 3] = 2.0 * d
    return out


def hess_s() -> np.ndarray:
    """d2 s_k / dx2 (6, 12, 12): 2I on the (a,a),(b,b) blocks, -2I on (a,b),(b,a)."""
    out = np.zeros((6, 12, 12))
    I3 = np.eye(3)
    for k, (a, b) in enumerate(LOCAL_EDGES):
        out[k, 3 * a:3 * a + 3, 3 * a:3 * a + 3] = 2 * I3
        out[k, 3 * b:3 * b + 3, 3 * b:3 * b + 3] = 2 * I3
        out[k, 3 * a:3 * a + 3, 3 * b:3 * b + 3] = -2 * I3
        out[k, 3 * b:3 * b + 3, 3 * a:3 * a + 3] = -2 * I3
    return out


def element_energy(x, tets, V, D2, q, lam, mu, chi=None, energy: str = "stvk") -> np.ndarray:
    """chi_e V_e Psi_e (Eq. 25 with Eq. 37 or Eq. 35), per tet."""
    if energy == "stvk":
        s = squared_edge_lengths(x, tets)
        C = cauchy_green_lsq(s, D2, q)
        psi = V * stvk_density(C, lam, mu)
    else:
        psi = V * edge_derivatives(x, tets, D2, q, lam, mu, energy)[0]
    return psi if chi is None else chi * psi


def element_forces(x, tets, V, D2, q, lam, mu, chi=None, energy: str = "stvk") -> np.ndarray:
    """Restoring nodal forces of every tet (t, 4, 3) by Eq. 12, times chi (Eq. 32):
    f_i = 2 V chi sum_{j != i} g_ij (x_j - x_i)."""
    _, g, _, _ = edge_derivatives(x, tets, D2, q, lam, mu, energy)
    P = x[np.asarray(tets, np.int64)]
    f = np.zeros_like(P)
    for k, (a, b) in enumerate(LOCAL_EDGES):
        w = (2.0 * V * g[:, k])[:, None]
        f[:, a] += w * (P[:, b] - P[:, a])
        f[:, b] += w * (P[:, a] - P[:, b])
    if chi is not None:
        f *= chi[:, None, None]
    return f


def element_tangent(x, tets, V, D2, q, lam, mu, chi=None, energy: str = "stvk") -> np.ndarray:
    """12x12 element tangent (Eq. 10 / Eq. 33), i.e. the Hessian of V Psi in the
    node positions: V [ sum_kl H_kl ds_k ds_l^T + sum_k g_k d2 s_k ], times chi."""
    _, g, H, _ = edge_derivatives(x, tets, D2, q, lam, mu, energy)
    Gs = grad_s(x, tets)
    K = np.einsum("tkl,tka,tlb->tab", H, Gs, Gs) + np.einsum("tk,kab->tab", g, hess_s())
    K *= V[:, None, None]
    if chi is not None:
        K *= chi[:, None, None]
    return K

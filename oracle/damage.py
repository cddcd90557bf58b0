"""Edge damage: stress, edge-normal projection, non-local average, relabel, chi.

Paper passages followed (Sec. 3.3-3.4):
* Eq. 14: the six Cartesian stress components [xx, yy, zz, xy, xz, yz].
  Reading: the symmetric second Piola-Kirchhoff stress S = 2 dPsi/dC (the
  printed "Piola-Kirchhoff" tensor must be symmetric to have six components).
* Eq. 16-19: normal stress along edge mn,
  sigma_mn = sum_i S_ii c_i^2 + kappa * sum_{i<j} S_ij c_i c_j, with the direction
  cosines c of the CURRENT edge (Eq. 17).  kappa = 2 is the tensor identity
  n.S.n (default); kappa = 1 is the formula as printed (option).
* Eq. 20: sigma*_mn = [T (sum_{|r - r0| <= R_d} w(r - r0) sigma_c(r))]_mn over
  tet centroids.  Readings: rest centroids (fixed neighbour sets), weight
  w = V_j (1 - r^2/R_d^2)^2 normalised to sum 1; R_d = 0 is the tet alone;
  the averaged field is chi_j S_j (option: raw S_j).
* Eq. 21: zeta = 1 (broken) when sigma* >= sigma_thres, never repaired (text
  after Eq. 21).  Readings: one zeta per mesh edge, driven by the maximum of
  sigma* over the tets sharing the edge; driver = sigma*/E (dimensionless,
  default) or sigma* (stress mode).
* Eq. 22-23 with the text: a broken edge's normal stress becomes zero, i.e.
  sigma' = (1 - zeta) sigma_f.
* Eq. 25: chi = sum |sigma'| / sum |sigma|, using the tet's own local sigma_f;
  chi = 0 when the element falls into two or more disjoint pieces (the unbroken
  edges no longer connect its 4 nodes); chi = 1 with no broken edge;
  chi = (unbroken edges)/6 when sum |sigma| <= 1e-12 E (0/0 guard).
"""
from __future__ import annotations

import numpy as np

from .mesh import LOCAL_EDGES

VOIGT = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def stress_voigt(C: np.ndarray, lam: float, mu: float, energy: str = "stvk", J=None) -> np.ndarray:
    """S = 2 dPsi/dC in Eq. 14 order.  Eq. 37: lam/2 (I_C - 3) Id + mu (C - Id).
    Eq. 35 (squared reading, signed J): mu (1 - 1/(I_C + 1)) Id + lam (J - a) J C^-1,
    from dJ/dC = J/2 C^-1."""
    I = np.trace(C, axis1=-2, axis2=-1)
    if energy == "stvk":
        S = lam / 2.0 * (I - 3.0)[..., None, None] * np.eye(3) + mu * (C - np.eye(3))
    else:
        a = 1.0 + mu / lam - mu / (4.0 * lam)
        S = (mu * (1.0 - 1.0 / (I + 1.0)))[..., None, None] * np.eye(3) \
            + (lam * (J - a) * J)[..., None, None] * np.linalg.inv(C)
    return np.stack([S[..., i, j] for i, j in VOIGT], -1)


def projection_T(x: np.ndarray, tets: np.ndarray, shear_coef: float = 2.0) -> np.ndarray:
    """Eq. 19 matrix T (t, 6, 6): row mn = [cx^2, cy^2, cz^2, k cx cy, k cx cz, k cy cz]
    with c the current unit vector of local edge mn (Eq. 17)."""
    P = x[np.asarray(tets, np.int64)]
    T = np.zeros((P.shape[0], 6, 6))
    for k, (a, b) in enumerate(LOCAL_EDGES):
        d = P[:, b] - P[:, a]
        c = d / np.linalg.norm(d, axis=1)[:, None]
        T[:, k, 0] = c[:, 0] ** 2
        T[:, k, 1] = c[:, 1] ** 2
        T[:, k, 2] = c[:, 2] ** 2
        T[:, k, 3] = shear_coef * c[:, 0] * c[:, 1]
        T[:, k, 4] = shear_coef * c[:, 0] * c[:, 2]
        T[:, k, 5] = shear_coef * c[:, 1] * c[:, 2]
    return T


def nonlocal_weights(centroids: np.ndarray, V: np.ndarray, nbrs, radius: float, subset=None):
    """Normalised Eq. 20 weights w_ej = V_j (1 - r^2/R^2)^2 / sum, one array per e."""
    idx = np.arange(len(centroids)) if subset is None else np.asarray(subset, np.int64)
    out = []
    for e, js in zip(idx, nbrs):
        if radius <= 0.0:
            out.append(np.ones(1))
            continue
        r2 = ((centroids[js] - centroids[e]) ** 2).sum(1)
        w = V[js] * (1.0 - r2 / radius ** 2) ** 2
        out.append(w / w.sum())
    return out


def nonlocal_average(sig_in: np.ndarray, nbrs, weights) -> np.ndarray:
    """The sum inside Eq. 20: sum_j w_ej sigma_c(j), one row per listed tet."""
    return np.stack([(w[:, None] * sig_in[js]).sum(0) for js, w in zip(nbrs, weights)])


def edge_driver(sig_star: np.ndarray, tet_edges: np.ndarray, n_edges: int, young: float,
                mode: str = "strain") -> np.ndarray:
    """Per-edge driver = max over incident tets of sigma*_mn (Eq. 20), divided by E
    in strain mode.  Edges with no incident tet get -inf."""
    drv = np.full(n_edges, -np.inf)
    np.maximum.at(drv, tet_edges.ravel(), sig_star.ravel())
    return drv / young if mode == "strain" else drv


def relabel(labels: np.ndarray, driver: np.ndarray, threshold: float) -> np.ndarray:
    """Eq. 21 plus irreversibility: zeta_new = zeta_old or (driver >= threshold)."""
    return (labels.astype(bool) | (driver >= threshold)).astype(np.uint8)


def tet_disconnected(broken6) -> bool:
    """True when the tet's unbroken edges leave its 4 nodes in >= 2 pieces."""
    adj = {v: set() for v in range(4)}
    for k, (a, b) in enumerate(LOCAL_EDGES):
        if not broken6[k]:
            adj[a].add(b)
            adj[b].add(a)
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) < 4


def chi(labels: np.ndarray, tet_edges: np.ndarray, sigf_local: np.ndarray, young: float) -> np.ndarray:
    """Energy degradation of Eq. 25 for every tet."""
    zeta = labels[tet_edges].astype(bool)                 # (t, 6)
    out = np.ones(tet_edges.shape[0])
    for e in np.nonzero(zeta.any(1))[0]:
        if tet_disconnected(zeta[e]):
            out[e] = 0.0
            continue
        den = np.abs(sigf_local[e]).sum()
        if den <= 1e-12 * young:
            out[e] = (~zeta[e]).sum() / 6.0
        else:
            out[e] = np.abs(np.where(zeta[e], 0.0, sigf_local[e])).sum() / den
    return out

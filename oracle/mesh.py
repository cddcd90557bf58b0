"""Mesh precompute for the oracle (Sec. 3.1-3.3).

The computational mesh is a graph whose vertices are the mesh nodes and whose
edges are the tet edges (Sec. 1, Sec. 3.2).  Edges are numbered as the sorted
list of unique (min, max) node pairs.  A tet's local edges follow the order of
Eq. 15: (1,2) (1,3) (1,4) (2,3) (2,4) (3,4), i.e. local node pairs
(0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
"""
from __future__ import annotations

import numpy as np

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def edges_of(tets: np.ndarray):
    """Unique sorted edges and the tet->edge map.

    Returns (edges (ne, 2) int64 with edges[:,0] < edges[:,1], lexicographic;
    tet_edges (t, 6) int64, global edge id of each local edge of Eq. 15).
    """
    tets = np.asarray(tets, np.int64)
    pairs = np.stack([tets[:, [a, b]] for a, b in LOCAL_EDGES], 1)   # (t, 6, 2)
    pairs = np.sort(pairs, axis=2)
    flat = pairs.reshape(-1, 2)
    edges, inv = np.unique(flat, axis=0, return_inverse=True)
    return edges, inv.reshape(-1, 6)


def rest_geometry(X: np.ndarray, tets: np.ndarray):
    """Rest volume V_e, rest squared edge lengths (D_mn)^2 and unit rest edge
    directions q_mn of every tet (Eq. 12, Eq. 27, Eq. 28).

    Local edge (m, n) points from local node m to local node n.
    """
    P = X[np.asarray(tets, np.int64)]                                  # (t, 4, 3)
    ev = np.stack([P[:, b] - P[:, a] for a, b in LOCAL_EDGES], 1)      # (t, 6, 3)
    D2 = np.einsum("tki,tki->tk", ev, ev)
    q = ev / np.sqrt(D2)[:, :, None]
    Dm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 2)
    V = np.abs(np.linalg.det(Dm)) / 6.0
    return V, D2, q


def lumped_mass(X: np.ndarray, tets: np.ndarray, rho: float, V: np.ndarray):
    """Row-sum lumped version of the element mass of Eq. 5: each node gets a
    quarter of rho*V_e from every tet it belongs to."""
    m = np.zeros(X.shape[0])
    np.add.at(m, np.asarray(tets, np.int64).ravel(), np.repeat(rho * V / 4.0, 4))
    return m


# Keast's 4-point rule on the reference tet (degree 2, so exact for the
# products N_a N_b of linear shape functions): barycentric points (a, b, b, b)
# and permutations, equal weights 1/4 of the volume.
_QA = 0.5854101966249685
_QB = 0.1381966011250105


def consistent_mass_blocks(tets: np.ndarray, rho: float, V: np.ndarray) -> np.ndarray:
    """Element mass of Eq. 5, m_e = int rho N_e^T N_e over the tet, as its
    scalar 4x4 node-pair table (the 12x12 matrix is this (x) I_3, Eq. 8):
    m_e[a, b] = rho V_e sum_q w_q N_a(p_q) N_b(p_q) by the 4-point rule.
    Returns (t, 4, 4)."""
    pts = np.full((4, 4), _QB)
    np.fill_diagonal(pts, _QA)                  # row q = barycentric point q = (N_0..N_3)(p_q)
    w = np.full(4, 0.25)
    ref = np.einsum("q,qa,qb->ab", w, pts, pts)   # int N_a N_b / V over the tet
    return rho * V[:, None, None] * ref[None]


def consistent_mass_matrix(X: np.ndarray, tets: np.ndarray, rho: float, V: np.ndarray):
    """Global mass of Eq. 4-5 with the consistent element masses, as a scipy
    CSR (3n x 3n) matrix m (x) I_3."""
    import scipy.sparse as sp
    tets = np.asarray(tets, np.int64)
    me = consistent_mass_blocks(tets, rho, V)
    n = X.shape[0]
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    m = sp.coo_matrix((me.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    return sp.kron(m, sp.identity(3), format="csr")


def centroids(X: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Rest centroid r of every tet (the r, r_0 of Eq. 20)."""
    return X[np.asarray(tets, np.int64)].mean(1)


def nonlocal_neighbours(X: np.ndarray, tets: np.ndarray, radius: float, brute: bool | None = None,
                        subset: np.ndarray | None = None):
    """For each tet e (or each e in ``subset``), the tets j whose rest centroid
    lies within ||r_j - r_e|| <= R_d (the summation range of Eq. 20), as a list
    of sorted index arrays.  R_d = 0 gives only the tet itself (Sec. 3.3: the
    local criterion).

    Small meshes use a brute-force distance matrix; larger ones a k-d tree
    range query (scipy), which returns the same sets.
    """
    r = centroids(X, tets)
    idx = np.arange(len(r)) if subset is None else np.asarray(subset, np.int64)
    if radius <= 0.0:
        return [np.array([e], np.int64) for e in idx]
    if brute is None:
        brute = len(r) * len(idx) <= 2.0e7
    if brute:
        out = []
        for e in idx:
            d = np.sqrt(((r - r[e]) ** 2).sum(1))
            out.append(np.nonzero(d <= radius)[0])
        return out
    from scipy.spatial import cKDTree
    tree = cKDTree(r)
    lists = tree.query_ball_point(r[idx], radius)
    return [np.array(sorted(lst), np.int64) for lst in lists]


def edge_incident_tets(tet_edges: np.ndarray, n_edges: int):
    """For each edge, the (tet, local edge) pairs that contain it."""
    t, k = np.nonzero(np.ones_like(tet_edges, bool))
    e = tet_edges[t, k]
    order = np.argsort(e, kind="stable")
    e, t, k = e[order], t[order], k[order]
    starts = np.searchsorted(e, np.arange(n_edges + 1))
    return starts, t, k

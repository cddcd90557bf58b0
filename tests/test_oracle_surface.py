"""Pins of the oracle's split visualisation mesh (Sec. 4.1, Fig. 6), no GPU.

* No broken edge: every entity's children sit at its current centroid.
* The face case Sec. 4.1 works through: with edges (1,2), (1,3) of face
  (1,2,3) broken and (2,3) whole, child 1 follows parent 1 and children 2, 3
  follow the average of parents 2 and 3 (written out here from the text).
* All six edges of a tet broken: each child follows its own parent.
* Quads: two per (tet, broken local edge), and every vertex of an a-side
  quad is a child of node a.
"""
import numpy as np

from oracle import mesh, surface
from workloads import beam_config, single_tet


def moved(X, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    return X + amp * rng.normal(size=X.shape)


def test_no_broken_edge_puts_children_at_current_centroids():
    w = beam_config()
    edges, _ = mesh.edges_of(w.tets)
    x = moved(w.nodes)
    V, Q, faces, tf = surface.surface(w.nodes, x, w.tets, edges, np.zeros(len(edges), np.uint8))
    N, NE, NF = len(x), len(edges), len(faces)
    assert len(Q) == 0
    np.testing.assert_allclose(V[:N], x)
    mid = x[edges].mean(1)
    np.testing.assert_allclose(V[N:N + 2 * NE].reshape(NE, 2, 3), np.repeat(mid[:, None], 2, 1), atol=1e-13)
    fc = x[faces].mean(1)
    np.testing.assert_allclose(V[N + 2 * NE:N + 2 * NE + 3 * NF].reshape(NF, 3, 3), np.repeat(fc[:, None], 3, 1),
                               atol=1e-13)
    tc = x[w.tets].mean(1)
    np.testing.assert_allclose(V[N + 2 * NE + 3 * NF:].reshape(-1, 4, 3), np.repeat(tc[:, None], 4, 1), atol=1e-13)


def test_worked_face_example_of_section_4_1():
    """Face (P1, P2, P3) = local nodes (0, 1, 2) of one tet; edges P1P2 and
    P1P3 broken, P2P3 whole."""
    X, tets = single_tet()
    x = moved(X, seed=1, amp=0.1)
    edges, _ = mesh.edges_of(tets)
    lab = np.zeros(len(edges), np.uint8)
    for a, b in ((0, 1), (0, 2)):
        lab[[k for k, e in enumerate(edges) if tuple(e) == (a, b)][0]] = 1
    V, Q, faces, tf = surface.surface(X, x, tets, edges, lab)
    f = [i for i, tri in enumerate(faces) if tuple(tri) == (0, 1, 2)][0]
    base = len(X) + 2 * len(edges) + 3 * f
    c = X[[0, 1, 2]].mean(0)
    d = x - X
    np.testing.assert_allclose(V[base + 0], c + d[0], atol=1e-15)
    np.testing.assert_allclose(V[base + 1], c + (d[1] + d[2]) / 2, atol=1e-15)
    np.testing.assert_allclose(V[base + 2], c + (d[1] + d[2]) / 2, atol=1e-15)
    # the broken edge P1P2 separates its two children; the whole edge P2P3 does not
    e12 = [k for k, e in enumerate(edges) if tuple(e) == (0, 1)][0]
    e23 = [k for k, e in enumerate(edges) if tuple(e) == (1, 2)][0]
    n = len(X)
    assert np.linalg.norm(V[n + 2 * e12] - V[n + 2 * e12 + 1]) > 1e-3
    np.testing.assert_allclose(V[n + 2 * e23], V[n + 2 * e23 + 1], atol=1e-15)
    # two broken local edges, two quads each
    assert len(Q) == 4


def test_fully_broken_tet_children_follow_their_parents():
    X, tets = single_tet()
    x = moved(X, seed=2, amp=0.1)
    edges, _ = mesh.edges_of(tets)
    V, Q, faces, tf = surface.surface(X, x, tets, edges, np.ones(len(edges), np.uint8))
    o2 = len(X) + 2 * len(edges) + 3 * len(faces)
    c = X.mean(0)
    np.testing.assert_allclose(V[o2:o2 + 4], c + (x - X), atol=1e-15)
    assert len(Q) == 12


def test_quads_belong_to_the_pieces_of_their_side():
    w = beam_config()
    edges, tet_edges = mesh.edges_of(w.tets)
    rng = np.random.default_rng(3)
    lab = (rng.random(len(edges)) < 0.05).astype(np.uint8)
    V, Q, faces, tf = surface.surface(w.nodes, moved(w.nodes, 4), w.tets, edges, lab)
    assert len(Q) == 2 * int(lab[tet_edges].sum())
    N, NE, NF = len(w.nodes), len(edges), len(faces)

    def parent(v):
        if v < N + 2 * NE:
            e, s = divmod(v - N, 2)
            return int(edges[e, s])
        if v < N + 2 * NE + 3 * NF:
            f, c = divmod(v - N - 2 * NE, 3)
            return int(faces[f, c])
        t, a = divmod(v - N - 2 * NE - 3 * NF, 4)
        return int(w.tets[t, a])

    owners = np.array([[parent(v) for v in q] for q in Q])
    assert (owners == owners[:, :1]).all()

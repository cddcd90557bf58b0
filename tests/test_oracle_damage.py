"""Pins of the oracle's damage part (no GPU): the hand-worked two-tet relabel of
Fig. 4, the local limit of Eq. 20, invariance of the normalised average on a
uniform field, monotone relabelling, and the disconnection rule of Eq. 25
against a library connected-components routine."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from oracle import damage, mesh
from oracle.mesh import LOCAL_EDGES
from oracle.step import Material, Model
from workloads import beam_config, two_tet_fig4

GOLD = os.path.join(os.path.dirname(__file__), "golden", "two_tet_fig4.json")


@pytest.mark.parametrize("radius", [0.0, 10.0])
@pytest.mark.parametrize("shear", [2.0, 1.0])
def test_two_tet_fig4_hand_worked(radius, shear):
    g = json.load(open(GOLD))
    X, tets = two_tet_fig4()
    x = X.copy()
    x[:, 0] *= g["stretch"]
    for case in g["cases"]:
        m = Model(X, tets, Material(g["young"], g["poisson"], 1000.0, threshold=case["threshold"],
                                    radius=radius, shear_coef=shear))
        assert [list(e) for e in m.edges] == g["edges"]
        st = m.rest_state()
        st.x = x
        drv, labels, chi, _ = m.damage_update(st)
        np.testing.assert_allclose(drv, g["driver"], rtol=1e-10)
        names = [g["edge_names"][i] for i in np.nonzero(labels)[0]]
        assert names == case["broken"]
        for e in range(2):
            assert damage.tet_disconnected(labels[m.tet_edges[e]].astype(bool)) == case["disconnected"][e]
        np.testing.assert_allclose(chi, case["chi"], rtol=1e-12, atol=0)


def test_local_limit_and_uniform_field():
    """R_d = 0 gives the tet's own stress (Sec. 3.3); a uniform field is unchanged
    by the normalised average for any R_d."""
    w = beam_config()
    X, tets = w.nodes, w.tets.astype(np.int64)
    cen = mesh.centroids(X, tets)
    V, _, _ = mesh.rest_geometry(X, tets)
    rng = np.random.default_rng(0)
    sig = rng.normal(size=(len(tets), 6))
    n0 = mesh.nonlocal_neighbours(X, tets, 0.0)
    w0 = damage.nonlocal_weights(cen, V, n0, 0.0)
    np.testing.assert_array_equal(damage.nonlocal_average(sig, n0, w0), sig)
    for R in (1.0, 1.5, 3.0):
        nb = mesh.nonlocal_neighbours(X, tets, R)
        wt = damage.nonlocal_weights(cen, V, nb, R)
        assert all(abs(ww.sum() - 1) < 1e-14 for ww in wt)
        uni = np.tile(rng.normal(size=6), (len(tets), 1))
        np.testing.assert_allclose(damage.nonlocal_average(uni, nb, wt), uni, rtol=1e-13)
        # every tet is its own neighbour, and neighbourhoods are symmetric
        assert all(e in set(nb[e]) for e in range(len(tets)))
        pairs = {(e, j) for e in range(len(tets)) for j in nb[e]}
        assert all((j, e) in pairs for (e, j) in pairs)


def test_neighbours_kdtree_equals_bruteforce():
    w = beam_config()
    a = mesh.nonlocal_neighbours(w.nodes, w.tets, 1.5, brute=True)
    b = mesh.nonlocal_neighbours(w.nodes, w.tets, 1.5, brute=False)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_relabel_is_monotone():
    rng = np.random.default_rng(1)
    labels = (rng.uniform(size=1000) < 0.2).astype(np.uint8)
    drv = rng.uniform(size=1000)
    new = damage.relabel(labels, drv, 0.7)
    assert np.all(new >= labels)
    np.testing.assert_array_equal(new, (labels == 1) | (drv >= 0.7))


def test_disconnection_rule_against_connected_components():
    """Eq. 25: chi = 0 iff the unbroken edges leave the tet's 4 nodes in >= 2
    pieces; checked for all 64 broken-edge masks with scipy's csgraph."""
    for mask in range(64):
        broken = [(mask >> k) & 1 == 1 for k in range(6)]
        rows = [a for k, (a, b) in enumerate(LOCAL_EDGES) if not broken[k]]
        cols = [b for k, (a, b) in enumerate(LOCAL_EDGES) if not broken[k]]
        G = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(4, 4))
        ncomp, _ = connected_components(G, directed=False)
        assert damage.tet_disconnected(broken) == (ncomp >= 2), mask


def test_chi_rules():
    """No broken edge -> 1; a broken edge zeroes exactly its own |sigma| share."""
    labels = np.zeros(6, np.uint8)
    tet_edges = np.arange(6)[None, :]
    sig = np.array([[1.0, -2.0, 3.0, 4.0, -5.0, 6.0]])
    assert damage.chi(labels, tet_edges, sig, 1.0)[0] == 1.0
    labels[1] = 1
    assert damage.chi(labels, tet_edges, sig, 1.0)[0] == pytest.approx(19.0 / 21.0)
    # 0/0 guard
    assert damage.chi(labels, tet_edges, np.zeros((1, 6)), 1.0)[0] == pytest.approx(5.0 / 6.0)


def test_edge_projection_is_quadratic_form():
    """Eq. 16-19 with shear coefficient 2 equal n.S.n for a symmetric S and the
    unit edge direction n (textbook normal traction); coefficient 1 is the
    formula as printed and differs by the shear part."""
    rng = np.random.default_rng(5)
    X = rng.normal(size=(4, 3))
    tets = np.array([[0, 1, 2, 3]])
    Svec = rng.normal(size=6)
    S = np.array([[Svec[0], Svec[3], Svec[4]], [Svec[3], Svec[1], Svec[5]], [Svec[4], Svec[5], Svec[2]]])
    T2 = damage.projection_T(X, tets, 2.0)[0]
    T1 = damage.projection_T(X, tets, 1.0)[0]
    for k, (a, b) in enumerate(LOCAL_EDGES):
        n = (X[b] - X[a]) / np.linalg.norm(X[b] - X[a])
        assert T2[k] @ Svec == pytest.approx(n @ S @ n, rel=1e-13, abs=1e-13)
        assert T1[k] @ Svec == pytest.approx(n @ np.diag(np.diag(S)) @ n + (n @ S @ n - n @ np.diag(np.diag(S)) @ n) / 2,
                                            rel=1e-12, abs=1e-12)


def test_shared_edge_takes_max_over_tets():
    """An edge shared by a strained and an unstrained tet takes the larger
    sigma* (one zeta per edge, driven by its most stressed tet)."""
    X, tets = two_tet_fig4()
    x = X.copy()
    x[4] += np.array([0.3, 0.25, 0.2])          # only BCDE deforms
    m2 = Model(X, tets, Material(1e6, 0.3, 1000.0, threshold=np.inf))
    st = m2.rest_state()
    st.x = x
    drv, _, _, sig_star = m2.damage_update(st)
    per_tet = []
    for e in range(2):
        me = Model(X, tets[e:e + 1], Material(1e6, 0.3, 1000.0, threshold=np.inf))
        se = me.rest_state()
        se.x = x
        d, _, _, _ = me.damage_update(se)
        per_tet.append({tuple(me.edges[i]): d[i] for i in range(len(me.edges))})
    for i, (a, b) in enumerate(m2.edges):
        vals = [pt[(a, b)] for pt in per_tet if (a, b) in pt]
        assert drv[i] == pytest.approx(max(vals), rel=1e-13)
    # the shared edges really see two different values
    shared = [i for i, (a, b) in enumerate(m2.edges) if all((a, b) in pt for pt in per_tet)]
    assert len(shared) == 3
    assert any(abs(per_tet[0][tuple(m2.edges[i])] - per_tet[1][tuple(m2.edges[i])]) > 1e-3 for i in shared)


def test_average_is_continuous_in_radius():
    """The weight vanishes at r = R_d, so a tet entering the ball changes the
    average only to second order in the radius increment."""
    w = beam_config()
    X, tets = w.nodes, w.tets.astype(np.int64)
    cen = mesh.centroids(X, tets)
    V, _, _ = mesh.rest_geometry(X, tets)
    e = 700
    d = np.sqrt(((cen - cen[e]) ** 2).sum(1))
    d_sorted = np.unique(d)
    r0 = d_sorted[40]                              # a centroid distance
    rng = np.random.default_rng(2)
    sig = rng.normal(size=(len(tets), 6))
    def jump(delta):
        vals = []
        for R in (r0 - delta, r0 + delta):
            nb = mesh.nonlocal_neighbours(X, tets, R, subset=[e])
            wt = damage.nonlocal_weights(cen, V, nb, R, subset=[e])
            vals.append(damage.nonlocal_average(sig, nb, wt)[0])
        return np.abs(vals[0] - vals[1]).max()

    # no O(1) jump as the tet at distance r0 enters: the change shrinks with delta
    j5, j6 = jump(1e-5), jump(1e-6)
    assert j6 < 1e-5
    assert 5.0 < j5 / j6 < 20.0

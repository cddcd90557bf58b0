"""Hand-worked pins of two oracle readings of Eq. 20 (Sec. 3.3).

* The weight: w_ej = V_j (1 - r^2/R_d^2)^2 over REST centroids, normalised.
* The chi lag: the averaged field is chi_j S_j with the chi of the previous
  step (the one stored in the state).

``tests/golden/nonlocal_chi_lag.json`` holds the hand-derived weights, drivers,
labels and chi of a four-tet case over two damage updates (exact fractions in
``tests/golden/derive_nonlocal_chi_lag.py``).  Beside the pins, each plausible
misreading is planted in the oracle here, on the CPU, and must fail them:
a dropped V_j, (1 - r/R_d)^2, current centroids, the raw S_j, chi recomputed
at the current positions, and the chi of the step's own relabel.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import damage, mesh
from oracle.step import Material, Model

GOLD = os.path.join(os.path.dirname(__file__), "golden", "nonlocal_chi_lag.json")
RTOL = 1e-10
ORACLE_WEIGHTS = damage.nonlocal_weights


@pytest.fixture(scope="module")
def gold():
    return json.load(open(GOLD))


def geometry(g):
    """Rest nodes and tets: corner, +x, +y, +z leg per tet (positive volume)."""
    nodes, tets = [], []
    for k, (o, a) in enumerate(zip(g["corners"], g["legs"])):
        o = np.array(o)
        nodes += [o, o + [a, 0, 0], o + [0, a, 0], o + [0, 0, a]]
        tets.append([4 * k, 4 * k + 1, 4 * k + 2, 4 * k + 3])
    return np.array(nodes), np.array(tets, np.int32)


def positions(g, X, step):
    """x = o + F (X - o) + t for every tet (homogeneous stretch about its corner)."""
    x = X.copy()
    for k, (f, t) in enumerate(zip(g[f"stretch_step{step}"], g["translate"])):
        rows = slice(4 * k, 4 * k + 4)
        o = X[4 * k]
        x[rows] = o + (X[rows] - o) * np.array(f) + np.array(t)
    return x


def model(g, **kw):
    X, tets = geometry(g)
    mat = Material(g["young"], g["poisson"], 1000.0, threshold=g["threshold"], radius=g["radius"], **kw)
    return X, Model(X, tets, mat)


def two_updates(g, m, X, chi_for_step2=None):
    """Damage updates at the step-1 and step-2 positions; returns both results."""
    st = m.rest_state()
    st.x = positions(g, X, 1)
    d1, l1, c1, _ = m.damage_update(st)
    st.labels, st.chi = l1, c1 if chi_for_step2 is None else chi_for_step2(m, l1, c1)
    st.x = positions(g, X, 2)
    d2, l2, c2, _ = m.damage_update(st)
    return (d1, l1, c1), (d2, l2, c2)


def close(a, b):
    return np.allclose(a, b, rtol=RTOL, atol=1e-14)


def test_weights_hand_worked(gold):
    X, m = model(gold)
    assert [list(map(int, n)) for n in m.nbrs] == [sorted(map(int, w)) for w in gold["weights"]]
    for e, w in enumerate(gold["weights"]):
        want = [float(Fraction(w[str(j)])) for j in m.nbrs[e]]
        np.testing.assert_allclose(m.weights[e], want, rtol=1e-13)


def test_two_steps_hand_worked(gold):
    X, m = model(gold)
    (d1, l1, c1), (d2, l2, c2) = two_updates(gold, m, X)
    for k, (d, l, c) in enumerate(((d1, l1, c1), (d2, l2, c2)), 1):
        ref = gold[f"step{k}"]
        np.testing.assert_allclose(d, ref["driver"], rtol=RTOL, atol=1e-14)
        np.testing.assert_array_equal(l, ref["broken"])
        np.testing.assert_allclose(c, ref["chi"], rtol=RTOL)
    # the case exercises what it pins: a tet with chi < 1 from step 1 enters
    # step 2's average, and step 2 breaks an edge that step 1 left whole
    assert 0.0 < c1.min() < 1.0
    assert (l2 > l1).any()


def test_sigma_bar_hand_worked(gold):
    """The weighted sum of Eq. 20 itself (before the projection T) at step 1."""
    X, m = model(gold)
    S, _, _ = m.stresses(positions(gold, X, 1))
    sbar = damage.nonlocal_average(S, m.nbrs, m.weights)
    want = np.array(gold["step1"]["sigma_bar_diag"])
    np.testing.assert_allclose(sbar[:, :3], want, rtol=RTOL)
    np.testing.assert_allclose(sbar[:, 3:], 0.0, atol=1e-15)


# ---- planted misreadings: each must miss the hand-worked values -------------

def _weights_without_volume(centroids, V, nbrs, radius, subset=None):
    return ORACLE_WEIGHTS(centroids, np.ones_like(V), nbrs, radius, subset)


def _weights_linear_distance(centroids, V, nbrs, radius, subset=None):
    idx = np.arange(len(centroids)) if subset is None else np.asarray(subset, np.int64)
    out = []
    for e, js in zip(idx, nbrs):
        r = np.sqrt(((centroids[js] - centroids[e]) ** 2).sum(1))
        w = V[js] * (1.0 - r / radius) ** 2
        out.append(w / w.sum())
    return out


@pytest.mark.parametrize("planted", [_weights_without_volume, _weights_linear_distance])
def test_planted_weight_mistakes_fail(gold, monkeypatch, planted):
    monkeypatch.setattr(damage, "nonlocal_weights", planted)
    X, m = model(gold)
    (d1, _, _), _ = two_updates(gold, m, X)
    assert not close(d1, gold["step1"]["driver"])


def test_planted_current_centroids_fail(gold):
    """Neighbour sets and weights taken from the CURRENT centroids at each update."""
    X, m = model(gold)
    R = gold["radius"]

    class CurrentCentroids(Model):
        def damage_update(self, state):
            cur = mesh.centroids(state.x, self.tets)
            self.nbrs = [np.nonzero(np.sqrt(((cur - cur[e]) ** 2).sum(1)) <= R)[0] for e in range(len(cur))]
            self.weights = damage.nonlocal_weights(cur, self.V, self.nbrs, R)
            return super().damage_update(state)

    mc = CurrentCentroids(X, m.tets, m.mat)
    (d1, _, _), (d2, _, _) = two_updates(gold, mc, X)
    assert not close(d1, gold["step1"]["driver"])
    assert not close(d2, gold["step2"]["driver"])


def test_planted_raw_stress_fails_at_step2(gold):
    """Averaging the raw S_j (the literal option) agrees at step 1 (all chi = 1)
    and misses step 2, where a degraded tet enters the average."""
    X, m = model(gold, average_degraded=False)
    (d1, _, _), (d2, _, _) = two_updates(gold, m, X)
    assert close(d1, gold["step1"]["driver"])
    assert not close(d2, gold["step2"]["driver"])


def test_planted_chi_at_current_positions_fails(gold):
    """chi recomputed from the stored labels at step 2's positions instead of
    the chi stored by step 1."""
    X, m = model(gold)
    x2 = positions(gold, X, 2)
    _, (d2, _, _) = two_updates(gold, m, X, chi_for_step2=lambda mm, l1, c1: mm.chi_from_labels(x2, l1))
    assert not close(d2, gold["step2"]["driver"])


def test_planted_new_chi_fails(gold):
    """The chi of step 2's own relabel used in step 2's average."""
    X, m = model(gold)
    _, (_, l2, c2) = two_updates(gold, m, X)
    st = m.rest_state()
    st.x = positions(gold, X, 1)
    _, l1, _, _ = m.damage_update(st)
    st.x, st.labels, st.chi = positions(gold, X, 2), l1, c2
    d2_new, _, _, _ = m.damage_update(st)
    assert not close(d2_new, gold["step2"]["driver"])

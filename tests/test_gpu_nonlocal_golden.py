"""The CUDA damage update against the hand-worked Eq. 20 values (Sec. 3.3).

The four-tet case of ``tests/golden/nonlocal_chi_lag.json``: rational weights
from unequal volumes and rest-centroid distances at R_d = 2, and a second
damage update whose average takes the chi stored by the first.  Each damage
update is the first phase of a step; the state is set before it, so the
drivers, labels and chi read back after the step are those of the update.
FP64 path at 1e-9, the mixed path at 1e-5 (its Eq. 20 sums are FP32).
"""
import json
import os

import numpy as np
import pytest

from test_oracle_nonlocal_golden import geometry, positions

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "nonlocal_chi_lag.json")


@pytest.mark.parametrize("precision,rtol", [(gf.FP64, 1e-9), (gf.MIXED, 1e-5)])
def test_damage_updates_match_hand_worked_values(precision, rtol):
    g = json.load(open(GOLD))
    X, tets = geometry(g)
    mat = gf.material(g["young"], g["poisson"], 1000.0, threshold=g["threshold"], radius=g["radius"])
    m = gf.mesh_create(X, tets, mat, precision=precision, cg_rtol=1e-10)
    assert [list(e) for e in m.edges_get()] == [[4 * k + a, 4 * k + b] for k in range(4)
                                                 for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))]
    zeros = np.zeros(X.size)
    dt = 1e-6
    # update 1 from the rest labels and chi = 1
    m.state_set(x=positions(g, X, 1).ravel(), v=zeros, labels=np.zeros(24, np.uint8), chi=np.ones(4))
    s = m.step(dt)
    assert s["status"] == 0
    drv, lab = m.damage_get()
    ref = g["step1"]
    np.testing.assert_allclose(drv, ref["driver"], rtol=rtol, atol=1e-12)
    np.testing.assert_array_equal(lab, ref["broken"])
    np.testing.assert_allclose(m.chi_get(), ref["chi"], rtol=rtol)
    # update 2 at the second positions with the labels and chi of update 1
    m.state_set(x=positions(g, X, 2).ravel(), v=zeros, labels=np.array(ref["broken"], np.uint8),
                chi=np.array(ref["chi"]))
    s = m.step(dt)
    assert s["status"] == 0
    drv, lab = m.damage_get()
    ref = g["step2"]
    np.testing.assert_allclose(drv, ref["driver"], rtol=rtol, atol=1e-12)
    np.testing.assert_array_equal(lab, ref["broken"])
    np.testing.assert_allclose(m.chi_get(), ref["chi"], rtol=rtol)
    assert s["n_broken"] == sum(ref["broken"])
    m.close()

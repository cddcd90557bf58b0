"""GPU parity of the stable Neo-Hookean energy (Eq. 35, squared reading,
signed J) against the oracle, through the C ABI.

The GPU element works from the deformation gradient (P and the closed-form
contraction of d2Psi/dF2); the oracle works in squared edge lengths (C by
Eq. 31, J = sgn sqrt(det C)).  The two are the same function for
non-degenerate tets, so the FP64 bar applies: 1e-9 relative element-wise on
drivers, the assembled system and the right-hand side, 1e-9 norm-wise on
velocities, positions within 1e-9 of each node's displacement, labels equal
outside the 1e-6 threshold band.
"""
import math

import numpy as np
import pytest

from helpers import (assert_close, assert_labels, assert_norm_close, assert_positions_close, block_values_from_csr,
                     deformed_state, gpu_material, oracle_model)
from workloads import beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def snh_mesh(w, precision=gf.FP64, **kw):
    mat = gpu_material(gf, w, **kw)
    mat.energy = gf.ENERGY_SNH
    return gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=1e-13, cg_maxit=20000)


def check_step(m, model, st, w, dt, pinned, pv=None, newton=1):
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
    stats = m.step(dt, w.f_ext.ravel(), pinned, pv)
    new, info = model.step(st, dt, w.f_ext, pinned, pv, newton_iters=newton)
    assert stats["status"] == 0 and stats["rel_res"] <= 1e-12
    drv, lab = m.damage_get()
    assert_close(drv, info["driver"], what="driver", floor=0.0, abs_floor=1e-13)
    assert_labels(lab, info["labels"], info["driver"], model.mat.threshold)
    same = np.array_equal(lab, info["labels"])
    if same:
        assert_close(m.chi_get(), info["chi"], floor=1e-12, what="chi")
        if newton == 1:
            rp, col, val, rhs = m.system_get()
            assert_close(val, block_values_from_csr(info["A"], rp, col), what="A blocks")
            assert_close(rhs, info["b"], what="rhs", abs_floor=1e-12 * dt * w.young * float(np.mean(model.D2)))
        assert_norm_close(m.velocities_get(), new.v, what="v")
        assert_positions_close(m.positions_get(), new.x, st.x, what="x")
    return new, info, stats, same


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.3, 1e-3)])
def test_snh_fracturing_steps_match_oracle(alpha, beta):
    w = beam_config()
    st = deformed_state(w, seed=31, amp=0.08)
    model0 = oracle_model(w, threshold=math.inf, energy="snh", alpha=alpha, beta=beta)
    drv0, *_ = model0.damage_update(st)
    theta = float(np.quantile(drv0, 0.95))
    model = oracle_model(w, threshold=theta, energy="snh", alpha=alpha, beta=beta)
    m = snh_mesh(w, threshold=theta, alpha=alpha, beta=beta)
    pv = np.tile([0.0, 0.05, 0.0], (len(w.pinned), 1))
    agreed = 0
    for _ in range(3):
        st, info, stats, same = check_step(m, model, st, w, w.dt, w.pinned, pv)
        agreed += same
        assert stats["n_broken"] > 0
    assert agreed >= 2


def test_snh_newton_iterations_match_oracle():
    w = beam_config()
    model = oracle_model(w, threshold=math.inf, energy="snh", mass="consistent")
    mat = gpu_material(gf, w, threshold=math.inf)
    mat.energy = gf.ENERGY_SNH
    mat.mass_matrix = gf.MASS_CONSISTENT
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-13, cg_maxit=20000)
    m.newton_set(4)
    st = deformed_state(w, seed=32, amp=0.1)
    new, info, stats, same = check_step(m, model, st, w, 5e-3, w.pinned, newton=4)
    assert same and stats["newton_iters"] == 4


def test_snh_with_inverted_tets_matches_oracle():
    """A few tets pushed through their opposite face (J < 0): the GPU's F route
    and the oracle's signed-J edge route agree on the restoring response."""
    w = beam_config()
    st = deformed_state(w, seed=33, amp=0.02, vamp=0.0)
    x = st.x.copy()
    free = np.setdiff1d(np.arange(w.n_nodes), w.pinned)
    rng = np.random.default_rng(3)
    flipped = []
    for t in rng.choice(w.n_tets, 40, replace=False):
        p = x[w.tets[t]]
        if w.tets[t, 3] not in free or w.tets[t, 3] in [w.tets[f, 3] for f in flipped]:
            continue
        n = np.cross(p[1] - p[0], p[2] - p[0])
        n /= np.linalg.norm(n)
        cand = x.copy()
        cand[w.tets[t, 3]] = p[3] - 1.3 * np.dot(p[3] - p[0], n) * n
        x = cand
        flipped.append(t)
        if len(flipped) == 4:
            break
    st.x = x
    from oracle import elastic
    sgn = elastic.orientation(x, w.tets, oracle_model(w, threshold=math.inf).q)
    assert (sgn < 0).sum() >= 4
    model = oracle_model(w, threshold=math.inf, energy="snh")
    m = snh_mesh(w, threshold=math.inf)
    new, info, stats, same = check_step(m, model, st, w, 1e-3, w.pinned)
    assert same


def test_snh_options_that_are_not_built_are_refused():
    w = beam_config()
    mat = gpu_material(gf, w)
    mat.energy = gf.ENERGY_SNH
    with pytest.raises(gf.GraphFEMError):
        gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED)
    m = gf.mesh_create(w.nodes, w.tets, mat)
    m.tuning_set(gf.graphfem.ASSEMBLY_COLOUR)
    with pytest.raises(gf.GraphFEMError):
        m.step(w.dt, w.f_ext.ravel(), w.pinned)
    bad = gpu_material(gf, w)
    bad.energy = gf.ENERGY_SNH
    bad.poisson = 0.0
    with pytest.raises(gf.GraphFEMError):
        gf.mesh_create(w.nodes, w.tets, bad)

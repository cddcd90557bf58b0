"""gf_mesh_autotune: the single-mesh autotuner times each candidate schedule
(FP64: gather or colour-ordered assembly x three-kernel, Chronopoulos-Gear or
nested solve; mixed: the two-kernel, three-kernel or persistent solve) on the
mesh's state, restored after each trial.  The state afterwards is the state
before, bit for bit; the mesh keeps the chosen tuning; and its next step gives
the bits of a fresh mesh stepped from the same state with that tuning.
"""
import math

import numpy as np
import pytest

from helpers import deformed_state, gpu_material, oracle_model
from workloads import beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def snapshot(m):
    return m.positions_get(), m.velocities_get(), m.damage_get()[1], m.chi_get()


@pytest.mark.parametrize("precision", [gf.FP64, gf.MIXED])
def test_autotune_keeps_state_and_picks_a_schedule(precision):
    w = beam_config()
    st = deformed_state(w, seed=43)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    mat = gpu_material(gf, w, threshold=float(np.quantile(d0, 0.95)))
    m = gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=1e-10, cg_maxit=20000)
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
    m.step(w.dt, w.f_ext.ravel(), w.pinned)   # some broken edges and chi < 1 in the saved state
    before = snapshot(m)
    best, ms = m.autotune(w.dt, w.f_ext.ravel(), w.pinned, trial_steps=2)
    assert ms > 0 and best == m.tuning_get()
    forms = (gf.SOLVE_CG, gf.SOLVE_KERNELS, gf.SOLVE_PERSISTENT) if precision == gf.MIXED else \
        (gf.SOLVE_KERNELS, gf.SOLVE_CG, gf.SOLVE_NESTED)
    assert best["solve_loop"] in forms
    for a, b in zip(snapshot(m), before):
        np.testing.assert_array_equal(a, b)
    fresh = gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=1e-10, cg_maxit=20000)
    fresh.tuning_set(**best)
    x, v, lab, chi = before
    fresh.state_set(x=x, v=v, labels=lab, chi=chi)
    sa = m.step(w.dt, w.f_ext.ravel(), w.pinned)
    sb = fresh.step(w.dt, w.f_ext.ravel(), w.pinned)
    assert sa["status"] == 0 and sa == sb
    np.testing.assert_array_equal(m.velocities_get(), fresh.velocities_get())
    m.close()
    fresh.close()


def test_autotune_refusals():
    w = beam_config()
    m = gf.mesh_create(w.nodes, w.tets, gpu_material(gf, w))
    with pytest.raises(gf.GraphFEMError) as e:
        m.autotune(w.dt, w.f_ext.ravel(), w.pinned, trial_steps=0)
    assert e.value.status == 1
    m.newton_set(2)
    with pytest.raises(gf.GraphFEMError) as e:
        m.autotune(w.dt, w.f_ext.ravel(), w.pinned)
    assert e.value.status == 8
    m.close()

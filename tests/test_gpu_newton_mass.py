"""GPU parity of the consistent mass (Eq. 5) and of Newton iterations on the
backward-Euler residual, against the oracle (through the C ABI).

FP64 bar as in the other parity tests: 1e-9 relative element-wise on the
assembled system and the drivers, 1e-9 norm-wise on velocities, positions
within 1e-9 of each node's displacement.  The GPU solves each Newton system
to 1e-13; the oracle solves exactly.  Mixed precision (consistent mass only):
1e-5 norm-wise on the velocity change.
"""
import math

import numpy as np
import pytest

from helpers import (assert_close, assert_norm_close, assert_positions_close, block_values_from_csr,
                     deformed_state, gpu_material, oracle_model)
from workloads import beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def make(w, mass, precision=gf.FP64, rtol=1e-13, **kw):
    mat = gpu_material(gf, w, **kw)
    mat.mass_matrix = gf.MASS_CONSISTENT if mass == "consistent" else gf.MASS_LUMPED
    return gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=rtol, cg_maxit=20000)


def set_state(m, st):
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)


@pytest.mark.parametrize("assembly", [gf.graphfem.ASSEMBLY_GATHER, gf.graphfem.ASSEMBLY_COLOUR], ids=["gather", "colour"])
@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.4, 2e-3)])
def test_consistent_mass_step_matches_oracle(assembly, alpha, beta):
    w = beam_config()
    st = deformed_state(w, seed=21)
    model0 = oracle_model(w, threshold=math.inf, alpha=alpha, beta=beta, mass="consistent")
    drv0, *_ = model0.damage_update(st)
    theta = float(np.quantile(drv0, 0.95))
    model = oracle_model(w, threshold=theta, alpha=alpha, beta=beta, mass="consistent")
    m = make(w, "consistent", threshold=theta, alpha=alpha, beta=beta)
    m.tuning_set(assembly=assembly)
    set_state(m, st)
    vp = np.tile([0.0, 0.05, 0.0], (len(w.pinned), 1))
    stats = m.step(w.dt, w.f_ext.ravel(), w.pinned, vp)
    new, info = model.step(st, w.dt, w.f_ext, w.pinned, vp)
    assert stats["status"] == 0 and stats["rel_res"] <= 1e-12 and stats["newton_iters"] == 1
    _, lab = m.damage_get()
    assert np.array_equal(lab, info["labels"]) and lab.sum() > 0
    rp, col, val, rhs = m.system_get()
    assert_close(val, block_values_from_csr(info["A"], rp, col), what="A blocks")
    assert_close(rhs, info["b"], what="rhs", abs_floor=1e-12 * w.dt * w.young * float(np.mean(model.D2)))
    assert_norm_close(m.velocities_get(), new.v, what="v")
    assert_positions_close(m.positions_get(), new.x, st.x, what="x")


def test_consistent_mass_mixed_precision_matches_oracle():
    w = beam_config()
    st = deformed_state(w, seed=22)
    model = oracle_model(w, threshold=math.inf, mass="consistent")
    m = make(w, "consistent", precision=gf.MIXED, rtol=1e-10, threshold=math.inf)
    set_state(m, st)
    stats = m.step(w.dt, w.f_ext.ravel(), w.pinned)
    new, info = model.step(st, w.dt, w.f_ext, w.pinned)
    assert stats["status"] == 0
    dv_gpu = m.velocities_get().reshape(-1, 3) - st.v
    assert np.linalg.norm(dv_gpu - info["dv"]) <= 1e-5 * np.linalg.norm(info["dv"])


@pytest.mark.parametrize("mass", ["lumped", "consistent"])
def test_newton_iterations_match_oracle(mass):
    """Three Newton iterations per step on a strongly deformed beam with damping
    and prescribed pinned velocities, two steps in a row (the second from the
    GPU's own state), against the oracle's Newton loop."""
    w = beam_config()
    kw = dict(alpha=0.2, beta=1e-3)
    model = oracle_model(w, threshold=math.inf, mass=mass, **kw)
    m = make(w, mass, threshold=math.inf, **kw)
    m.newton_set(3)
    st = deformed_state(w, seed=23, amp=0.08)
    set_state(m, st)
    vp = np.tile([0.0, 0.1, 0.0], (len(w.pinned), 1))
    dt = 5e-3
    for _ in range(2):
        stats = m.step(dt, w.f_ext.ravel(), w.pinned, vp)
        new, info = model.step(st, dt, w.f_ext, w.pinned, vp, newton_iters=3)
        assert stats["status"] == 0 and stats["newton_iters"] == 3 and stats["rel_res"] <= 1e-12
        assert_norm_close(m.velocities_get(), new.v, what="v")
        assert_positions_close(m.positions_get(), new.x, st.x, what="x")
        st = new
    # the iterations matter: one linearised step lands elsewhere
    one, _ = model.step(st, dt, w.f_ext, w.pinned, vp)
    more, _ = model.step(st, dt, w.f_ext, w.pinned, vp, newton_iters=3)
    assert np.linalg.norm(one.v - more.v) > 1e-6 * np.linalg.norm(more.v - st.v)


def test_newton_stops_on_its_tolerance():
    w = beam_config()
    model = oracle_model(w, threshold=math.inf)
    m = make(w, "lumped", threshold=math.inf)
    m.newton_set(12, 1e-9)
    st = deformed_state(w, seed=24, amp=0.08)
    set_state(m, st)
    stats = m.step(5e-3, w.f_ext.ravel(), w.pinned)
    assert stats["status"] == 0 and 2 <= stats["newton_iters"] < 12
    new, info = model.step(st, 5e-3, w.f_ext, w.pinned, newton_iters=12)
    assert_norm_close(m.velocities_get(), new.v, rtol=1e-8, what="v")


def test_newton_options_outside_the_fp64_single_mesh_path_are_refused():
    w = beam_config()
    mx = make(w, "lumped", precision=gf.MIXED)
    with pytest.raises(gf.GraphFEMError):
        mx.newton_set(2)
    m1, m2 = make(w, "lumped"), make(w, "lumped")
    m1.newton_set(2)
    b = gf.Batch([m1, m2])
    f = [torch.tensor(w.f_ext.ravel(), dtype=torch.float64, device="cuda")] * 2
    pins = [torch.tensor(w.pinned, dtype=torch.int32, device="cuda")] * 2
    with pytest.raises(gf.GraphFEMError):
        b.step(w.dt, f, pins)
    with pytest.raises(gf.GraphFEMError):
        m1.newton_set(0)

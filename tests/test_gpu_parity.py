"""GPU parity: the CUDA step (through the C ABI) against the CPU FP64 oracle.

Bar (FP64): every element within 1e-9 relative (with an absolute floor of 1e-12
of the array's scale for entries formed by cancellation), states within 1e-9
norm-wise, break labels identical except edges whose driver lies within 1e-6
of the threshold.  The GPU solves to 1e-13 here; the oracle solves exactly.
"""
import math

import numpy as np
import pytest

from helpers import (assert_close, assert_labels, assert_norm_close, assert_positions_close, block_values_from_csr,
                     deformed_state, gpu_material, oracle_model)
from oracle.step import State
from workloads import beam_config, single_tet

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def gpu_mesh(w, mat, rtol=1e-13):
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=rtol, cg_maxit=20000)
    return m


def gpu_state(m, st: State):
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)


def compare_step(m, model, st, w, dt, f_ext, pinned, pinned_vel=None, threshold=None):
    gpu_state(m, st)
    stats = m.step(dt, f_ext.ravel() if f_ext is not None else None, pinned, pinned_vel)
    new, info = model.step(st, dt, np.zeros_like(w.nodes) if f_ext is None else f_ext, pinned, pinned_vel)
    drv, lab = m.damage_get()
    finite = np.isfinite(info["driver"])
    # drivers are strains (or stresses): rounding noise of a state at rest is
    # ~1e-16 strain, so the absolute floor is 1e-13 strain (x E in stress mode)
    floor = 1e-13 * (model.mat.young if model.mat.driver_mode == "stress" else 1.0)
    assert_close(drv[finite], info["driver"][finite], what="driver", floor=0.0, abs_floor=floor)
    th = model.mat.threshold
    assert_labels(lab, info["labels"], info["driver"], th)
    same_labels = np.array_equal(lab, info["labels"])
    if same_labels:
        assert_close(m.chi_get(), info["chi"], floor=1e-12, what="chi")
        rp, col, val, rhs = m.system_get()
        assert_close(val, block_values_from_csr(info["A"], rp, col), what="A blocks")
        # rhs floor: the force of a 1e-12 strain, dt * E * h^2 * 1e-12 (rest-state rounding)
        assert_close(rhs, info["b"], what="rhs",
                     abs_floor=1e-12 * dt * model.mat.young * float(np.mean(model.D2)))
        assert_norm_close(m.velocities_get(), new.v, what="v")
        assert_positions_close(m.positions_get(), new.x, st.x, what="x")
    assert stats["rel_res"] <= 1e-12
    assert stats["n_broken"] == int(lab.sum())
    return new, info, stats, same_labels


def test_one_step_from_rest_beam():
    w = beam_config()
    model = oracle_model(w)
    m = gpu_mesh(w, gpu_material(gf, w))
    st = model.rest_state()
    new, info, stats, same = compare_step(m, model, st, w, w.dt, w.f_ext, w.pinned)
    assert same and stats["cg_iters"] > 0 and stats["n_broken"] == 0


VARIANTS = {
    "nonlocal_strain": dict(radius=1.5),
    "local_printed_shear_raw_avg": dict(radius=0.0, shear_coef=1.0, average_degraded=False),
    "stress_driver_damped": dict(radius=1.5, driver_mode="stress", alpha=0.5, beta=1e-3),
}


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fracturing_steps_from_deformed_state(name):
    """Three steps, each from the oracle's state (state_set), at a threshold that
    breaks ~5% of the edges per step; exercises Eq. 20-25 and chi-scaled assembly."""
    kw = dict(VARIANTS[name])
    w = beam_config()
    model0 = oracle_model(w, threshold=math.inf, **kw)
    st = deformed_state(w, seed=11)
    drv0, _, _, _ = model0.damage_update(st)
    theta = float(np.quantile(drv0[np.isfinite(drv0)], 0.95))
    model = oracle_model(w, threshold=theta, **kw)
    gkw = {k: v for k, v in kw.items() if k != "radius"}
    m = gpu_mesh(w, gpu_material(gf, w, threshold=theta, radius=kw["radius"], **gkw))
    rng = np.random.default_rng(5)
    pv = 0.05 * rng.normal(size=(len(w.pinned), 3))
    agreed = 0
    for k in range(3):
        new, info, stats, same = compare_step(m, model, st, w, w.dt, w.f_ext, w.pinned, pv)
        agreed += same
        assert stats["n_broken"] > 0
        st = new
    assert agreed >= 2
    assert (st.chi < 1).any()


def test_trajectory_beam_20_steps():
    """Full C1 run (20 steps, no resync): GPU and oracle stay within 1e-9."""
    w = beam_config()
    model = oracle_model(w)
    m = gpu_mesh(w, gpu_material(gf, w))
    st = model.rest_state()
    for k in range(w.steps):
        st, _ = model.step(st, w.dt, w.f_ext, w.pinned)
        m.step(w.dt, w.f_ext.ravel(), w.pinned)
    assert_positions_close(m.positions_get(), st.x, w.nodes, ulps=64.0, what="x after 20 steps")
    assert_norm_close(m.velocities_get(), st.v, what="velocity")


def test_single_tet_and_fully_pinned():
    X, tets = single_tet()
    from workloads import Workload
    w = Workload("one", X, tets, 1e5, 0.3, 1000.0, 1e-2, 1, math.inf, 0.0, np.zeros((4, 3)), np.array([0, 1, 2], np.int32))
    model = oracle_model(w)
    m = gpu_mesh(w, gpu_material(gf, w))
    st = model.rest_state()
    st.x = X + np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0], [0.05, -0.03, 0.1]])
    st.v = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0], [0.2, 0.1, -0.3]])
    f = np.zeros((4, 3))
    f[3] = [1.0, 2.0, -3.0]
    compare_step(m, model, st, w, w.dt, f, w.pinned)
    # every node pinned: dv is the prescribed change, no CG iteration
    gpu_state(m, st)
    pv = np.full((4, 3), 0.25)
    stats = m.step(w.dt, f.ravel(), np.arange(4, dtype=np.int32), pv)
    assert stats["cg_iters"] == 0
    np.testing.assert_allclose(m.velocities_get().reshape(4, 3), pv, rtol=0, atol=1e-15)


def test_rest_without_load_stays_put():
    w = beam_config()
    m = gpu_mesh(w, gpu_material(gf, w), rtol=1e-6)
    for _ in range(3):
        s = m.step(w.dt, None, w.pinned)
    assert np.abs(m.positions_get() - w.nodes.ravel()).max() < 1e-13
    assert s["n_broken"] == 0


def test_bad_arguments():
    w = beam_config()
    m = gpu_mesh(w, gpu_material(gf, w))
    with pytest.raises(gf.GraphFEMError):
        m.step(-1.0)
    with pytest.raises(gf.GraphFEMError):
        m.step(w.dt, None, np.array([0, 10**6], np.int32))
    with pytest.raises(ValueError):
        m.step(w.dt, np.zeros(5))


def test_deterministic_and_resume_bit_identical():
    w = beam_config()
    st0 = deformed_state(w, seed=3, amp=0.03)
    model = oracle_model(w, threshold=math.inf)
    d0, _, _, _ = model.damage_update(st0)
    theta = float(np.quantile(d0, 0.97))
    mat = gpu_material(gf, w, threshold=theta)

    def run(n, m=None):
        if m is None:
            m = gpu_mesh(w, mat, rtol=1e-8)
            gpu_state(m, st0)
        for _ in range(n):
            m.step(w.dt, w.f_ext.ravel(), w.pinned)
        return m

    a = run(4)
    b = run(4)
    np.testing.assert_array_equal(a.positions_get(), b.positions_get())
    np.testing.assert_array_equal(a.damage_get()[0], b.damage_get()[0])
    # checkpoint after 2 steps, resume on a fresh mesh
    c = run(2)
    ck = (c.positions_get(), c.velocities_get(), c.damage_get()[1], c.chi_get())
    d = gpu_mesh(w, mat, rtol=1e-8)
    d.state_set(x=ck[0], v=ck[1], labels=ck[2], chi=ck[3])
    run(2, d)
    np.testing.assert_array_equal(a.positions_get(), d.positions_get())
    np.testing.assert_array_equal(a.damage_get()[1], d.damage_get()[1])


def test_device_inputs_match_host_inputs():
    w = beam_config()
    mat = gpu_material(gf, w)
    a = gpu_mesh(w, mat, rtol=1e-10)
    b = gpu_mesh(w, mat, rtol=1e-10)
    a.step(w.dt, w.f_ext.ravel(), w.pinned)
    fd = torch.tensor(w.f_ext.ravel(), dtype=torch.float64, device="cuda")
    pd = torch.tensor(w.pinned, dtype=torch.int32, device="cuda")
    b.step(w.dt, fd, pd)
    np.testing.assert_array_equal(a.positions_get(), b.positions_get())
    xd = torch.empty(3 * w.n_nodes, dtype=torch.float64, device="cuda")
    b.positions_get(out=xd)
    np.testing.assert_array_equal(xd.cpu().numpy(), a.positions_get())


def test_assembly_schedules_agree():
    """Two-phase gather and colour-ordered scatter assemble the same system
    (up to summation order) and both match the oracle."""
    w = beam_config()
    model0 = oracle_model(w, threshold=math.inf)
    st = deformed_state(w, seed=17)
    d0, _, _, _ = model0.damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta)
    out = {}
    for sched in (gf.graphfem.ASSEMBLY_GATHER, gf.graphfem.ASSEMBLY_COLOUR):
        m = gpu_mesh(w, gpu_material(gf, w, threshold=theta))
        m.tuning_set(sched)
        assert m.tuning_get()["assembly"] == sched
        new, info, stats, same = compare_step(m, model, st, w, w.dt, w.f_ext, w.pinned)
        assert same
        out[sched] = (m.system_get()[2], m.velocities_get())
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-12, atol=1e-12 * np.abs(out[0][0]).max())
    assert np.linalg.norm(out[0][1] - out[1][1]) <= 1e-12 * np.linalg.norm(out[0][1])


def test_metrics_log_one_line_per_step(tmp_path):
    """The binding's per-step metrics log writes one JSON line per step with the
    step's statistics."""
    import json
    w = beam_config()
    m = gpu_mesh(w, gpu_material(gf, w), rtol=1e-8)
    log = tmp_path / "steps.jsonl"
    m.metrics_log(str(log))
    stats = [m.step(w.dt, w.f_ext.ravel(), w.pinned) for _ in range(3)]
    m.metrics_log(None)
    recs = [json.loads(line) for line in log.read_text().splitlines()]
    assert [r["step"] for r in recs] == [0, 1, 2]
    assert [r["cg_iters"] for r in recs] == [s["cg_iters"] for s in stats]
    assert all(r["status"] == 0 and r["dt"] == w.dt for r in recs)
    m.close()

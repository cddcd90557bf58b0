"""GPU tests of the persistent solve of the mixed-precision step.

The whole refinement loop (inner FP32 PCG, double-float residual) runs as one
cooperative launch with grid barriers between its phases.  Its phases do the
arithmetic of the kernel-by-kernel form (a lone mesh's phases group the rows
into at most one CTA set), so the two forms must agree to rounding and its
graph replay and stream launches to the last bit; the persistent form must match the FP64
oracle at the reduced-precision bar on a fracturing beam and on a stiff
(glass-like) beam with many inner iterations; a batch's members must step as
they do alone; and a barrier wait that runs out (a test hook makes one CTA
skip its arrival) must end the step with GF_TIMEOUT after about a second,
leaving the mesh usable once its state is set again.
"""
import math
import time

import numpy as np
import pytest

from helpers import assert_close, assert_labels, assert_norm_close, deformed_state, gpu_material, oracle_model
from test_gpu_batch import box_workloads, start_states
from workloads import Workload, beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

RTOL32, FLOOR32, BAND32 = 1e-5, 1e-6, 1e-5


def mixed_mesh(w, mat, rtol=1e-10, solve=gf.SOLVE_PERSISTENT, launch=gf.STEP_GRAPH):
    m = gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=rtol, cg_maxit=20000)
    m.tuning_set(step_launch=launch, solve_loop=solve)
    return m


def glass_beam():
    b = beam_config()
    return Workload("beam_glass", b.nodes, b.tets, 7e10, 0.22, 2500.0, 5e-4, 3, math.inf, 1.5,
                    b.f_ext * 20.0, b.pinned)


def test_persistent_agrees_with_kernel_form_and_graph_with_stream():
    """Fracturing beam steps: the persistent solve agrees with the kernel-by-kernel
    one (the same arithmetic; a lone mesh's phases take at most one CTA set, so
    the reductions group the rows differently) and its graph replay gives the
    same bits as its stream launches."""
    w = beam_config()
    st = deformed_state(w, seed=13)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    mat = gpu_material(gf, w, threshold=float(np.quantile(d0, 0.95)))
    a = mixed_mesh(w, mat, launch=gf.STEP_GRAPH)
    c = mixed_mesh(w, mat, launch=gf.STEP_STREAM)
    b = mixed_mesh(w, mat, solve=gf.SOLVE_KERNELS, launch=gf.STEP_STREAM)
    for m in (a, b, c):
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
    for k in range(4):
        sa = a.step(w.dt, w.f_ext.ravel(), w.pinned)
        sb = b.step(w.dt, w.f_ext.ravel(), w.pinned)
        sc = c.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert sa["status"] == 0 and sb["status"] == 0 and sc["status"] == 0
        assert sa == sc
        np.testing.assert_array_equal(a.velocities_get(), c.velocities_get())
        np.testing.assert_array_equal(a.damage_get()[1], c.damage_get()[1])
        assert_norm_close(a.velocities_get(), b.velocities_get(), rtol=1e-7, what=f"v, persistent vs kernels, step {k}")
        assert abs(sa["cg_iters"] - sb["cg_iters"]) <= 1
    assert sa["n_broken"] > 0


def test_persistent_fracturing_steps_match_oracle():
    w = beam_config()
    st = deformed_state(w, seed=17)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta)
    m = mixed_mesh(w, gpu_material(gf, w, threshold=theta))
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert s["status"] == 0 and s["rel_res"] <= 1e-10
        drv, lab = m.damage_get()
        assert_close(drv, info["driver"], rtol=RTOL32, floor=FLOOR32, what="driver (persistent)")
        assert_labels(lab, info["labels"], info["driver"], theta, band=BAND32)
        if np.array_equal(lab, info["labels"]):
            assert_norm_close(m.velocities_get(), new.v, rtol=RTOL32, what="v (persistent)")
        st = new


def test_persistent_stiff_glass_many_iterations():
    """Glass stiffness on the beam: tens of inner iterations per step inside one
    launch; each step from the oracle's state matches the oracle at 1e-5."""
    w = glass_beam()
    model = oracle_model(w)
    m = mixed_mesh(w, gpu_material(gf, w), rtol=1e-8)
    st = model.rest_state()
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, _ = model.step(st, w.dt, w.f_ext, w.pinned)
        assert s["status"] == 0 and s["rel_res"] <= 1e-8 and s["cg_iters"] > 10
        assert_norm_close(m.velocities_get(), new.v, rtol=RTOL32, what=f"v (glass, persistent, step {k})")
        st = new


def test_persistent_batch_members_step_as_alone():
    """A batch runs every member's solve in one cooperative launch whose phases
    take only the blocks of the meshes still iterating; each member steps bit
    for bit as it does alone, in graph and stream form."""
    ws = box_workloads()
    states, thetas = start_states(ws)
    for graph in (1, 0):
        singles, members = [], []
        for w, th in zip(ws, thetas):
            mat = gf.material(w.young, w.poisson, w.density, threshold=th, radius=w.radius)
            singles.append(gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=1e-10, cg_maxit=5000))
            singles[-1].tuning_set(solve_loop=gf.SOLVE_KERNELS)   # the three-kernel inner PCG of the phases
            members.append(gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=1e-10, cg_maxit=5000))
        for m, st in zip(singles + members, states + states):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
        b = gf.Batch(members)
        b.tuning_set(graph=graph, solve_loop=gf.SOLVE_PERSISTENT)
        f = [w.f_ext.ravel() for w in ws]
        pins = [w.pinned for w in ws]
        for _ in range(2):
            sb = b.step(ws[0].dt, f, pins)
            ss = [m.step(w.dt, w.f_ext.ravel(), w.pinned) for m, w in zip(singles, ws)]
            assert all(x["status"] == 0 for x in sb + ss)
            assert [x["cg_iters"] for x in sb] == [x["cg_iters"] for x in ss]
            assert len({x["cg_iters"] for x in sb}) > 1      # the members converge independently
            for ms, mb in zip(singles, members):
                np.testing.assert_array_equal(mb.velocities_get(), ms.velocities_get())
        b.close()
        for m in singles + members:
            m.close()


def test_barrier_wait_runs_out_and_mesh_recovers():
    """The test hook makes one CTA skip its first barrier arrival: every wait of
    that barrier runs out after about a second, the step returns GF_TIMEOUT, and
    the mesh steps correctly once its state is set again."""
    w = beam_config()
    mat = gpu_material(gf, w)
    ref = mixed_mesh(w, mat)
    m = mixed_mesh(w, mat)
    st = deformed_state(w, seed=5)
    for launch in (gf.STEP_STREAM, gf.STEP_GRAPH):
        m.tuning_set(step_launch=launch, solve_loop=gf.SOLVE_PERSISTENT, wait_test=1)
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
        t0 = time.perf_counter()
        with pytest.raises(gf.GraphFEMError) as e:
            m.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert e.value.status == 6          # GF_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        m.tuning_set(step_launch=launch, solve_loop=gf.SOLVE_PERSISTENT, wait_test=0)
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
        ref.state_set(x=st.x.ravel(), v=st.v.ravel())
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        r = ref.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert s["status"] == 0 and r["status"] == 0
        np.testing.assert_array_equal(m.velocities_get(), ref.velocities_get())

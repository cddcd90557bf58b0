"""GPU tests of the solver loops in the Chronopoulos-Gear form (GF_SOLVE_CG).

The form takes w = A z and the three dot products in one kernel and the
vector updates in another, one grid reduction per iteration; its iterates are
the three-kernel PCG's in exact arithmetic.  The FP64 PCG in this form must
match the FP64 oracle at 1e-9 on fracturing beam steps and on a stiff
(glass-like) beam with tens of iterations, agree with the three-kernel form,
and give the same bits in graph replay and stream launches.  The mixed path's
inner FP32 PCG in this form must meet the reduced-precision bar (1e-5) against
the oracle on the same two beams, with graph and stream bit-identical.  Forms a
precision does not support are refused.
"""
import math

import numpy as np
import pytest

from helpers import (assert_close, assert_labels, assert_norm_close, assert_positions_close, deformed_state,
                     gpu_material, oracle_model)
from workloads import Workload, beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def fp64_mesh(w, mat, launch, solve=gf.SOLVE_CG, rtol=1e-13):
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=rtol, cg_maxit=20000)
    m.tuning_set(step_launch=launch, solve_loop=solve)
    return m


@pytest.mark.parametrize("launch", [gf.STEP_GRAPH, gf.STEP_STREAM])
def test_cg_form_fracturing_steps_match_oracle(launch):
    w = beam_config()
    st = deformed_state(w, seed=23)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta)
    m = fp64_mesh(w, gpu_material(gf, w, threshold=theta), launch)
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert s["status"] == 0 and s["rel_res"] <= 1e-12 and s["cg_iters"] > 0
        drv, lab = m.damage_get()
        fin = np.isfinite(info["driver"])
        assert_close(drv[fin], info["driver"][fin], what="driver", floor=0.0, abs_floor=1e-13)
        assert_labels(lab, info["labels"], info["driver"], theta)
        if np.array_equal(lab, info["labels"]):
            assert_norm_close(m.velocities_get(), new.v, what="v (CG form)")
            assert_positions_close(m.positions_get(), new.x, st.x, what="x (CG form)")
        st = new


def test_cg_form_stiff_glass_beam():
    """Glass stiffness: tens of PCG iterations per step; the CG form reaches the
    same 1e-12 residual as the three-kernel form in about as many iterations,
    matches both it and the oracle's direct solve to the accuracy the residual
    allows, and gives the same bits in graph replay and stream launches."""
    b = beam_config()
    w = Workload("beam_glass", b.nodes, b.tets, 7e10, 0.22, 2500.0, 5e-4, 3, math.inf, 1.5, b.f_ext * 20.0, b.pinned)
    model = oracle_model(w)
    mat = gpu_material(gf, w)
    g = fp64_mesh(w, mat, gf.STEP_GRAPH)
    c = fp64_mesh(w, mat, gf.STEP_STREAM)
    k3 = fp64_mesh(w, mat, gf.STEP_GRAPH, solve=gf.SOLVE_KERNELS)
    st = model.rest_state()
    for k in range(3):
        for m in (g, c, k3):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
        sg = g.step(w.dt, w.f_ext.ravel(), w.pinned)
        sc = c.step(w.dt, w.f_ext.ravel(), w.pinned)
        sk = k3.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, _ = model.step(st, w.dt, w.f_ext, w.pinned)
        assert sg["status"] == 0 and sg["cg_iters"] > 10 and sg["rel_res"] <= 1e-12
        assert sg == sc
        np.testing.assert_array_equal(g.velocities_get(), c.velocities_get())
        assert abs(sg["cg_iters"] - sk["cg_iters"]) <= 2 and sk["rel_res"] <= 1e-12
        # both forms stop at a 1e-12 residual; on this stiff system the solution
        # error is the residual times the condition number (about 1e4), so the
        # comparison with the direct solve and between the forms is at 1e-7
        assert_norm_close(g.velocities_get(), new.v, rtol=1e-7, what=f"v (glass, CG form, step {k})")
        assert_norm_close(k3.velocities_get(), new.v, rtol=1e-7, what=f"v (glass, three kernels, step {k})")
        assert_norm_close(g.velocities_get(), k3.velocities_get(), rtol=1e-7, what="v, CG form vs three kernels")
        st = new


RTOL32, FLOOR32, BAND32 = 1e-5, 1e-6, 1e-5


def mixed_mesh(w, mat, launch, solve=gf.SOLVE_CG, rtol=1e-10):
    m = gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=rtol, cg_maxit=20000)
    m.tuning_set(step_launch=launch, solve_loop=solve)
    return m


def test_mixed_cg_form_fracturing_steps_match_oracle():
    """Mixed path, inner PCG in the two-kernel form: fracturing beam steps from
    the oracle's state meet the reduced-precision bar; graph replay and stream
    launches give the same bits."""
    w = beam_config()
    st = deformed_state(w, seed=29)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta)
    mat = gpu_material(gf, w, threshold=theta)
    g = mixed_mesh(w, mat, gf.STEP_GRAPH)
    c = mixed_mesh(w, mat, gf.STEP_STREAM)
    for k in range(3):
        for m in (g, c):
            m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        sg = g.step(w.dt, w.f_ext.ravel(), w.pinned)
        sc = c.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert sg["status"] == 0 and sg["rel_res"] <= 1e-10 and sg["cg_iters"] > 0
        assert sg == sc
        np.testing.assert_array_equal(g.velocities_get(), c.velocities_get())
        drv, lab = g.damage_get()
        assert_close(drv, info["driver"], rtol=RTOL32, floor=FLOOR32, what="driver (mixed, CG form)")
        assert_labels(lab, info["labels"], info["driver"], theta, band=BAND32)
        if np.array_equal(lab, info["labels"]):
            assert_norm_close(g.velocities_get(), new.v, rtol=RTOL32, what=f"v (mixed, CG form, step {k})")
        st = new


def test_mixed_cg_form_stiff_glass_beam():
    """Glass stiffness: tens of inner iterations per step.  The two-kernel inner
    form reaches the outer 1e-8 residual, matches the oracle at 1e-5 and the
    three-kernel inner form to the accuracy the residual allows, in about as
    many inner iterations."""
    b = beam_config()
    w = Workload("beam_glass", b.nodes, b.tets, 7e10, 0.22, 2500.0, 5e-4, 3, math.inf, 1.5, b.f_ext * 20.0, b.pinned)
    model = oracle_model(w)
    mat = gpu_material(gf, w)
    g = mixed_mesh(w, mat, gf.STEP_GRAPH, rtol=1e-8)
    k3 = mixed_mesh(w, mat, gf.STEP_GRAPH, solve=gf.SOLVE_KERNELS, rtol=1e-8)
    st = model.rest_state()
    for k in range(3):
        for m in (g, k3):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
        sg = g.step(w.dt, w.f_ext.ravel(), w.pinned)
        sk = k3.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, _ = model.step(st, w.dt, w.f_ext, w.pinned)
        assert sg["status"] == 0 and sg["cg_iters"] > 10 and sg["rel_res"] <= 1e-8
        assert sk["status"] == 0 and abs(sg["cg_iters"] - sk["cg_iters"]) <= max(4, sk["cg_iters"] // 10)
        assert_norm_close(g.velocities_get(), new.v, rtol=RTOL32, what=f"v (glass, mixed CG form, step {k})")
        assert_norm_close(g.velocities_get(), k3.velocities_get(), rtol=1e-5, what="v, mixed CG vs three kernels")
        st = new


@pytest.mark.parametrize("launch", [gf.STEP_GRAPH, gf.STEP_STREAM])
def test_fp64_nested_form_fracturing_steps_match_oracle(launch):
    """FP64 steps whose linear solve is the nested one (flexible FP64 PCG around
    an FP32 inner PCG): it stops at the FP64 residual test (1e-12 here), so the
    steps match the oracle at the FP64 bar."""
    w = beam_config()
    st = deformed_state(w, seed=31)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta)
    m = fp64_mesh(w, gpu_material(gf, w, threshold=theta), launch, solve=gf.SOLVE_NESTED)
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert s["status"] == 0 and s["rel_res"] <= 1e-12 and s["cg_iters"] > 0
        drv, lab = m.damage_get()
        fin = np.isfinite(info["driver"])
        assert_close(drv[fin], info["driver"][fin], what="driver", floor=0.0, abs_floor=1e-13)
        assert_labels(lab, info["labels"], info["driver"], theta)
        if np.array_equal(lab, info["labels"]):
            assert_norm_close(m.velocities_get(), new.v, what="v (nested form)")
            assert_positions_close(m.positions_get(), new.x, st.x, what="x (nested form)")
        st = new


def test_fp64_nested_form_stiff_glass_beam():
    """Glass stiffness: the nested form reaches the same 1e-12 FP64 residual as
    the three-kernel PCG and agrees with it and with the oracle's direct solve
    to the accuracy that residual allows (R36)."""
    b = beam_config()
    w = Workload("beam_glass", b.nodes, b.tets, 7e10, 0.22, 2500.0, 5e-4, 3, math.inf, 1.5, b.f_ext * 20.0, b.pinned)
    model = oracle_model(w)
    mat = gpu_material(gf, w)
    n = fp64_mesh(w, mat, gf.STEP_GRAPH, solve=gf.SOLVE_NESTED)
    k3 = fp64_mesh(w, mat, gf.STEP_GRAPH, solve=gf.SOLVE_KERNELS)
    st = model.rest_state()
    for k in range(3):
        for m in (n, k3):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
        sn = n.step(w.dt, w.f_ext.ravel(), w.pinned)
        sk = k3.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, _ = model.step(st, w.dt, w.f_ext, w.pinned)
        assert sn["status"] == 0 and sn["rel_res"] <= 1e-12 and sn["cg_iters"] > 10
        assert_norm_close(n.velocities_get(), new.v, rtol=1e-7, what=f"v (glass, nested form, step {k})")
        assert_norm_close(n.velocities_get(), k3.velocities_get(), rtol=1e-7, what="v, nested vs three kernels")
        st = new


def test_fp64_nested_form_with_newton_iterations():
    """Two Newton iterations per step: the second solve starts from the first
    one's dv (a warm start, the reference |b|^2 from k_pcg_init); the nested
    form matches the three-kernel PCG to its 1e-12 residual on fracturing beam
    steps."""
    w = beam_config()
    st = deformed_state(w, seed=37)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    mat = gpu_material(gf, w, threshold=float(np.quantile(d0, 0.95)))
    n = fp64_mesh(w, mat, gf.STEP_STREAM, solve=gf.SOLVE_NESTED)
    k3 = fp64_mesh(w, mat, gf.STEP_STREAM, solve=gf.SOLVE_KERNELS)
    for m in (n, k3):
        m.newton_set(2)
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
    for k in range(3):
        sn = n.step(w.dt, w.f_ext.ravel(), w.pinned)
        sk = k3.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert sn["status"] == 0 and sk["status"] == 0 and sn["newton_iters"] == 2 == sk["newton_iters"]
        assert sn["rel_res"] <= 1e-12
        np.testing.assert_array_equal(n.damage_get()[1], k3.damage_get()[1])
        assert_norm_close(n.velocities_get(), k3.velocities_get(), rtol=1e-9, what=f"v, nested vs kernels, step {k}")


def test_solve_forms_refused_where_not_built():
    w = beam_config()
    mat = gpu_material(gf, w)
    m64 = gf.mesh_create(w.nodes, w.tets, mat)
    with pytest.raises(gf.GraphFEMError) as e:
        m64.tuning_set(solve_loop=gf.SOLVE_PERSISTENT)
    assert e.value.status == 8
    m32 = gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED)
    with pytest.raises(gf.GraphFEMError) as e:
        m32.tuning_set(solve_loop=gf.SOLVE_NESTED)
    assert e.value.status == 8
    m64.close()
    m32.close()

"""GPU tests of batched stepping (many meshes per launch, CUDA-graph replay).

A batch step runs the same kernel bodies with the same per-mesh launch
geometry and reduction order as stepping each mesh alone, so the results must
be bit-identical; the meshes converge independently; graph replay and stream
launches agree; the autotuner leaves the state untouched; and one member is
checked against the CPU oracle.
"""
import math

import numpy as np
import pytest

from helpers import assert_norm_close, assert_positions_close, deformed_state, oracle_model
from workloads import Workload, jitter, kuhn_box

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def box_workloads(seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for k, (nx, nz) in enumerate([(2, 3), (3, 5), (4, 4), (2, 9), (5, 6)]):
        nodes, tets, grid = kuhn_box(nx, nx, nz)
        nodes = jitter(nodes, 0.01, 1.0, 100 + k)
        E = float(10 ** rng.uniform(4, 7))
        f = np.zeros_like(nodes)
        top = grid[:, 2] == nz
        f[top] = rng.normal(size=3) * E * 1e-4
        pinned = np.nonzero(grid[:, 2] == 0)[0].astype(np.int32)
        out.append(Workload(f"box{k}", nodes, tets, E, 0.3, 1000.0, 1e-3, 3, math.inf, 1.5, f, pinned))
    return out


def make(ws, precision, thetas):
    ms = []
    for w, th in zip(ws, thetas):
        mat = gf.material(w.young, w.poisson, w.density, threshold=th, radius=w.radius)
        ms.append(gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=1e-10, cg_maxit=5000))
    return ms


def start_states(ws):
    states, thetas = [], []
    for k, w in enumerate(ws):
        st = deformed_state(w, seed=40 + k, amp=0.03)
        d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
        states.append(st)
        thetas.append(float(np.quantile(d0, 0.95)))
    return states, thetas


@pytest.mark.parametrize("precision", [gf.FP64, gf.MIXED])
@pytest.mark.parametrize("graph", [1, 0])
def test_batch_equals_single_meshes(precision, graph):
    ws = box_workloads()
    states, thetas = start_states(ws)
    singles = make(ws, precision, thetas)
    members = make(ws, precision, thetas)
    for m1, m2, st in zip(singles, members, states):
        for m in (m1, m2):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
    batch = gf.Batch(members)
    batch.tuning_set(graph=graph, chunk=3)
    f = [w.f_ext.ravel() for w in ws]
    pins = [w.pinned for w in ws]
    for step in range(3):
        bstats = batch.step(1e-3, f, pins)
        sstats = [m.step(1e-3, w.f_ext.ravel(), w.pinned) for m, w in zip(singles, ws)]
        for k, (a, b) in enumerate(zip(bstats, sstats)):
            assert a["status"] == 0 and a["cg_iters"] == b["cg_iters"] and a["n_broken"] == b["n_broken"], (k, a, b)
            assert a["rel_res"] == b["rel_res"]
    for k, (m1, m2) in enumerate(zip(singles, members)):
        np.testing.assert_array_equal(m1.positions_get(), m2.positions_get(), err_msg=f"mesh {k}")
        np.testing.assert_array_equal(m1.damage_get()[1], m2.damage_get()[1])
    assert sum(s["n_broken"] for s in bstats) > 0
    assert batch.launch_count() > 0
    batch.close()


@pytest.mark.parametrize("precision", [gf.FP64, gf.MIXED])
@pytest.mark.parametrize("form,grid,graph", [(gf.SOLVE_KERNELS, 48, 1), (gf.SOLVE_DISTRIBUTED, 48, 1),
                                             (gf.SOLVE_DISTRIBUTED, 7, 0), (gf.SOLVE_DISTRIBUTED, 0, 1)],
                         ids=["budget-48", "distributed-48", "distributed-7-stream", "distributed-default"])
def test_batch_grid_budget(precision, form, grid, graph):
    """A grid budget (the loop kernels' CTAs split over the meshes by size), or
    the distributed loop (a fixed grid split over the meshes still iterating,
    from a work table rebuilt on the device each iteration; 7 CTAs make each
    CTA take many blocks), changes only the reductions' summation order:
    members agree with their single-mesh steps to rounding and converge to the
    same tolerance."""
    ws = box_workloads()
    states, thetas = start_states(ws)
    singles = make(ws, precision, thetas)
    members = make(ws, precision, thetas)
    for m1, m2, st in zip(singles, members, states):
        for m in (m1, m2):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
    batch = gf.Batch(members)
    batch.tuning_set(graph=graph, chunk=8, grid_budget=grid, solve_loop=form)
    assert batch.tuning_get()["grid_budget"] == grid and batch.tuning_get()["solve_loop"] == form
    f = [w.f_ext.ravel() for w in ws]
    pins = [w.pinned for w in ws]
    bstats = batch.step(1e-3, f, pins)
    sstats = [m.step(1e-3, w.f_ext.ravel(), w.pinned) for m, w in zip(singles, ws)]
    for a, b in zip(bstats, sstats):
        assert a["status"] == 0 and a["rel_res"] <= 1e-10 and b["rel_res"] <= 1e-10
    for m1, m2 in zip(singles, members):
        x1, x2 = m1.positions_get(), m2.positions_get()
        assert np.abs(x1 - x2).max() <= 1e-9 * np.abs(x1).max()
    batch.close()


@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("form,inner", [(gf.SOLVE_KERNELS, 1), (gf.SOLVE_KERNELS, 8), (gf.SOLVE_CG, 0),
                                        (gf.SOLVE_CG, 3)])
def test_batch_inner_pass_and_cg_form_step_as_alone(graph, form, inner):
    """Mixed batches with 1 to 8 inner iterations per loop pass, in the three-
    and two-kernel inner forms: each member steps bit for bit as the same mesh
    stepped alone in the same form (a member whose inner solve ends inside a
    pass only idles), over two fracturing steps."""
    ws = box_workloads()
    states, thetas = start_states(ws)
    singles = make(ws, gf.MIXED, thetas)
    members = make(ws, gf.MIXED, thetas)
    for m1, m2, st in zip(singles, members, states):
        m1.tuning_set(solve_loop=form)
        for m in (m1, m2):
            m.state_set(x=st.x.ravel(), v=st.v.ravel())
    batch = gf.Batch(members)
    batch.tuning_set(graph=graph, chunk=8, solve_loop=form, inner=inner)
    assert batch.tuning_get()["inner"] == inner
    f = [w.f_ext.ravel() for w in ws]
    pins = [w.pinned for w in ws]
    for _ in range(2):
        bstats = batch.step(1e-3, f, pins)
        sstats = [m.step(1e-3, w.f_ext.ravel(), w.pinned) for m, w in zip(singles, ws)]
        assert [x["cg_iters"] for x in bstats] == [x["cg_iters"] for x in sstats]
        assert all(x["status"] == 0 for x in bstats)
        for m1, m2 in zip(singles, members):
            np.testing.assert_array_equal(m2.velocities_get(), m1.velocities_get())
    batch.close()


def test_batch_tuning_refusals():
    ws = box_workloads()
    b64 = gf.Batch(make(ws, gf.FP64, [math.inf] * len(ws)))
    with pytest.raises(gf.GraphFEMError) as e:
        b64.tuning_set(solve_loop=gf.SOLVE_CG)
    assert e.value.status == 8
    b32 = gf.Batch(make(ws, gf.MIXED, [math.inf] * len(ws)))
    for bad in ({"inner": -1}, {"inner": 65}, {"solve_loop": 7}):
        with pytest.raises(gf.GraphFEMError) as e:
            b32.tuning_set(**bad)
        assert e.value.status == 1
    b64.close()
    b32.close()


def test_batch_meshes_converge_independently():
    ws = box_workloads(seed=5)
    ms = make(ws, gf.FP64, [math.inf] * len(ws))
    batch = gf.Batch(ms)
    stats = batch.step(1e-3, [w.f_ext.ravel() for w in ws], [w.pinned for w in ws])
    iters = [s["cg_iters"] for s in stats]
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-10 for s in stats)
    assert len(set(iters)) > 1, iters          # stiffness differs per mesh
    batch.close()


def test_batch_member_matches_oracle():
    ws = box_workloads(seed=7)
    states, thetas = start_states(ws)
    ms = make(ws, gf.FP64, thetas)
    for m, st in zip(ms, states):
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
    batch = gf.Batch(ms)
    batch.step(1e-3, [w.f_ext.ravel() for w in ws], [w.pinned for w in ws])
    k = 2
    w = ws[k]
    new, info = oracle_model(w, threshold=thetas[k]).step(states[k], 1e-3, w.f_ext, w.pinned)
    if np.array_equal(ms[k].damage_get()[1], info["labels"]):
        assert_norm_close(ms[k].velocities_get(), new.v, what="batched member v")
        assert_positions_close(ms[k].positions_get(), new.x, states[k].x, what="batched member x")
    batch.close()


def test_autotune_keeps_state_and_picks_a_schedule():
    ws = box_workloads(seed=9)
    ms = make(ws, gf.MIXED, [math.inf] * len(ws))
    ref = make(ws, gf.MIXED, [math.inf] * len(ws))
    batch = gf.Batch(ms)
    f = [w.f_ext.ravel() for w in ws]
    pins = [w.pinned for w in ws]
    before = [m.positions_get() for m in ms]
    best, ms_per_step = batch.autotune(1e-3, f, pins, trial_steps=2)
    assert best["graph"] in (0, 1) and ms_per_step > 0
    for m, x0 in zip(ms, before):
        np.testing.assert_array_equal(m.positions_get(), x0)
    batch.step(1e-3, f, pins)
    # members step bit for bit as alone when every mesh keeps its single-mesh
    # grid: in the chosen form, or for the persistent batch loop in the
    # three-kernel form (its sums are grouped as those kernels group them); a
    # budget or the distributed loop regroups the sums
    same_bits = best["grid_budget"] == 0 and best["solve_loop"] != gf.SOLVE_DISTRIBUTED
    single_form = {gf.SOLVE_PERSISTENT: gf.SOLVE_KERNELS}.get(best["solve_loop"], best["solve_loop"])
    for m, r, w in zip(ms, ref, ws):
        if best["solve_loop"] != gf.SOLVE_DISTRIBUTED:
            r.tuning_set(solve_loop=single_form)
        r.step(1e-3, w.f_ext.ravel(), w.pinned)
        if same_bits:
            np.testing.assert_array_equal(m.positions_get(), r.positions_get())
        else:
            x1, x2 = r.positions_get(), m.positions_get()
            assert np.abs(x1 - x2).max() <= 1e-9 * np.abs(x1).max()
    batch.close()


def test_bench_batch_configuration_members_match_singles_and_oracle():
    """The batch bench.py times (64 boxes of 2k-80k tets, mixed, CUDA graph):
    after two steps every member is bit-identical to the same mesh stepped
    alone, and the two smallest members match the FP64 oracle at the FP32
    tolerance (1e-5 norm-wise)."""
    from workloads import batch_configs
    ws = batch_configs()

    def mesh(w):
        mat = gf.material(w.young, w.poisson, w.density, threshold=w.threshold, radius=w.radius)
        return gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=1e-6)

    ms = [mesh(w) for w in ws]
    batch = gf.Batch(ms)
    assert batch.tuning_get()["graph"] == 1
    for _ in range(2):
        stats = batch.step(ws[0].dt, [w.f_ext.ravel() for w in ws], [w.pinned for w in ws])
        assert all(s["status"] == 0 and s["rel_res"] <= 1e-6 for s in stats)
    for k, w in enumerate(ws):
        single = mesh(w)
        for _ in range(2):
            single.step(w.dt, w.f_ext.ravel(), w.pinned)
        np.testing.assert_array_equal(ms[k].positions_get(), single.positions_get())
        np.testing.assert_array_equal(ms[k].velocities_get(), single.velocities_get())
        np.testing.assert_array_equal(ms[k].damage_get()[1], single.damage_get()[1])
        single.close()
    for k in np.argsort([w.n_tets for w in ws])[:2]:
        w = ws[k]
        model = oracle_model(w)
        st = model.rest_state()
        for _ in range(2):
            st, info = model.step(st, w.dt, w.f_ext, w.pinned)
        np.testing.assert_array_equal(ms[k].damage_get()[1], info["labels"])
        assert_norm_close(ms[k].velocities_get(), st.v, rtol=1e-5, what=f"batch member {k} v (mixed)")
    batch.close()

"""The plain step as one CUDA graph replay (GF_STEP_GRAPH, the default) against
the kernel-by-kernel stream form (GF_STEP_STREAM), through the C ABI.

Both run the same kernels in the same order on the same data, so the bar is
bit-identity: positions, velocities, drivers and labels over a fracturing
run, across the re-captures a changed dt or changed device input pointers
force, for the FP64 and the mixed-precision path.
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


def _fracturing_material(w):
    st = deformed_state(w, seed=23, amp=0.08)
    d0, _, _, _ = oracle_model(w, threshold=math.inf).damage_update(st)
    return st, gpu_material(gf, w, threshold=float(np.quantile(d0, 0.95)))


def _pair(w, mat, st, precision):
    out = []
    for launch in (gf.STEP_GRAPH, gf.STEP_STREAM):
        m = gf.mesh_create(w.nodes, w.tets, mat, precision=precision, cg_rtol=1e-8, cg_maxit=20000)
        m.tuning_set(step_launch=launch)
        assert m.tuning_get()["step_launch"] == launch
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
        out.append(m)
    return out


def _same(a, b):
    np.testing.assert_array_equal(a.positions_get(), b.positions_get())
    np.testing.assert_array_equal(a.velocities_get(), b.velocities_get())
    da, la = a.damage_get()
    db, lb = b.damage_get()
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(da, db)


@pytest.mark.parametrize("precision", [gf.FP64, gf.MIXED], ids=["fp64", "mixed"])
def test_graph_step_matches_stream_step(precision):
    w = beam_config()
    st, mat = _fracturing_material(w)
    g, s = _pair(w, mat, st, precision)
    broke = 0
    for k, dt in enumerate([w.dt, w.dt, 0.5 * w.dt, 0.5 * w.dt, w.dt]):   # dt changes force re-captures
        sg = g.step(dt, w.f_ext.ravel(), w.pinned)
        ss = s.step(dt, w.f_ext.ravel(), w.pinned)
        for key in ("status", "cg_iters", "n_broken", "n_new_broken", "n_chi_zero", "refine_sweeps"):
            assert sg[key] == ss[key], (k, key)
        assert sg["rel_res"] == ss["rel_res"]
        _same(g, s)
        broke = sg["n_broken"]
    assert broke > 0


def test_graph_step_device_inputs_and_pointer_change():
    """A new device input buffer every step (copied into the mesh's buffers by
    the graph form, read in place by the stream form) gives the same bits."""
    w = beam_config()
    st, mat = _fracturing_material(w)
    g, s = _pair(w, mat, st, gf.FP64)
    for k in range(3):
        fd = torch.tensor(w.f_ext.ravel() * (1.0 + 0.1 * k), dtype=torch.float64, device="cuda")   # new pointer
        pd = torch.tensor(w.pinned, dtype=torch.int32, device="cuda")
        g.step(w.dt, fd, pd)
        s.step(w.dt, fd, pd)
        torch.cuda.synchronize()
        _same(g, s)


def test_graph_step_launch_count_and_iteration_limit():
    """The launch count covers the replayed WHILE iterations, and the iteration
    cap still ends an unconverged solve with GF_CG_MAXITER."""
    w = beam_config()
    st, mat = _fracturing_material(w)
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-14, cg_maxit=3)
    m.state_set(x=st.x.ravel(), v=st.v.ravel())
    before = m.launch_count()
    with pytest.raises(gf.GraphFEMError) as e:
        m.step(w.dt, w.f_ext.ravel(), w.pinned)
    assert e.value.status == 4   # GF_CG_MAXITER
    assert m.launch_count() > before

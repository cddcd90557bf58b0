"""GPU parity of the mixed-precision step (FP32 tangents, stresses, non-local
average and inner PCG; FP64 state, iterative-refinement residual, dot products
and threshold test) against the CPU FP64 oracle.

Bar for reduced precision: 1e-5 relative (element-wise with a floor of 1e-6 of
the array's scale, i.e. ~16 FP32 roundings, for values formed by cancellation;
norm-wise for the state), the
FP64 residual of the linear solve at the requested tolerance, and break labels
identical except edges whose FP64 driver lies within 1e-5 of the threshold
(FP32 stresses carry ~1e-7 relative rounding, averaged over ~160 neighbours).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from helpers import (assert_close, assert_labels, assert_norm_close, assert_positions_close, block_values_from_csr,
                     deformed_state, gpu_material, oracle_model)
from workloads import beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

RTOL32 = 1e-5
FLOOR32 = 1e-6
BAND32 = 1e-5


def mixed_mesh(w, mat, rtol=1e-10):
    return gf.mesh_create(w.nodes, w.tets, mat, precision=gf.MIXED, cg_rtol=rtol, cg_maxit=20000)


@pytest.mark.parametrize("radius,avg", [(1.5, True), (0.0, False)])
def test_mixed_fracturing_steps_match_fp64_oracle(radius, avg):
    w = beam_config()
    model0 = oracle_model(w, threshold=math.inf, radius=radius, average_degraded=avg)
    st = deformed_state(w, seed=13)
    d0, _, _, _ = model0.damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta, radius=radius, average_degraded=avg)
    m = mixed_mesh(w, gpu_material(gf, w, threshold=theta, radius=radius, average_degraded=avg))
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        stats = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert stats["status"] == 0 and stats["rel_res"] <= 1e-10
        assert stats["refine_sweeps"] >= 1
        drv, lab = m.damage_get()
        assert_close(drv, info["driver"], rtol=RTOL32, floor=FLOOR32, what="driver (mixed)")
        assert_labels(lab, info["labels"], info["driver"], theta, band=BAND32)
        if np.array_equal(lab, info["labels"]):
            assert_close(m.chi_get(), info["chi"], rtol=RTOL32, floor=FLOOR32, what="chi (mixed)")
            rp, col, val, rhs = m.system_get()
            assert_close(val, block_values_from_csr(info["A"], rp, col), rtol=RTOL32, floor=FLOOR32, what="A32")
            assert_close(rhs, info["b"], rtol=RTOL32, floor=FLOOR32, what="rhs (mixed)")
            assert_norm_close(m.velocities_get(), new.v, rtol=RTOL32, what="v (mixed)")
            assert_positions_close(m.positions_get(), new.x, st.x, rtol=RTOL32, noise=1e-7, what="x (mixed)")
        st = new


def test_mixed_residual_is_fp64_accurate():
    """The refinement's residual is formed in FP64-level accuracy: recomputing
    ||b - A32 dv|| in float64 on the host from the GPU's own system agrees."""
    w = beam_config()
    m = mixed_mesh(w, gpu_material(gf, w, threshold=math.inf), rtol=1e-12)
    st = deformed_state(w, seed=2, amp=0.02)
    m.state_set(x=st.x.ravel(), v=st.v.ravel())
    s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
    rp, col, val, rhs = m.system_get()
    rows = np.repeat(np.arange(w.n_nodes), np.diff(rp))
    r3 = (3 * rows[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
    c3 = (3 * col[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
    A = sp.csr_matrix((val.ravel(), (r3.ravel(), c3.ravel())), shape=(3 * w.n_nodes,) * 2)
    dv = m.velocities_get() - st.v.ravel()
    free = np.ones(w.n_nodes, bool)
    free[w.pinned] = False
    fr = np.repeat(free, 3)
    dvp = dv.copy()
    dvp[fr] = 0
    ref = np.linalg.norm((rhs - A @ dvp)[fr])
    res = np.linalg.norm((rhs - A @ dv)[fr]) / ref
    assert res <= 1e-12 and s["rel_res"] <= 1e-12
    assert abs(res - s["rel_res"]) <= 1e-3 * res + 1e-14   # both at the rounding level here


def test_mixed_stiff_glass_material():
    """Glass-like stiffness (E = 7e10, rho = 2500) on the beam: many CG
    iterations.  Each step starts from the oracle's state, and the mixed step
    matches the oracle's step at the reduced-precision bar of 1e-5."""
    from workloads import Workload
    b = beam_config()
    w = Workload("beam_glass", b.nodes, b.tets, 7e10, 0.22, 2500.0, 5e-4, 3, math.inf, 1.5,
                 b.f_ext * 20.0, b.pinned)
    model = oracle_model(w)
    m = mixed_mesh(w, gpu_material(gf, w), rtol=1e-8)
    st = model.rest_state()
    for k in range(3):
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        new, info = model.step(st, w.dt, w.f_ext, w.pinned)
        assert s["status"] == 0 and s["rel_res"] <= 1e-8 and s["cg_iters"] > 10
        assert_norm_close(m.velocities_get(), new.v, rtol=RTOL32, what=f"v (glass, mixed, step {k})")
        assert_positions_close(m.positions_get(), new.x, st.x, rtol=RTOL32, noise=1e-7, what=f"x (glass, step {k})")
        st = new


def test_mixed_resume_bit_identical_and_rest():
    w = beam_config()
    mat = gpu_material(gf, w)
    a = mixed_mesh(w, mat, rtol=1e-8)
    for _ in range(3):
        a.step(w.dt, None, w.pinned)
    np.testing.assert_array_equal(a.positions_get(), w.nodes.ravel())   # no load: stays at rest
    b = mixed_mesh(w, mat, rtol=1e-8)
    c = mixed_mesh(w, mat, rtol=1e-8)
    for _ in range(4):
        b.step(w.dt, w.f_ext.ravel(), w.pinned)
    for _ in range(2):
        c.step(w.dt, w.f_ext.ravel(), w.pinned)
    d = mixed_mesh(w, mat, rtol=1e-8)
    d.state_set(x=c.positions_get(), v=c.velocities_get(), labels=c.damage_get()[1], chi=c.chi_get())
    for _ in range(2):
        d.step(w.dt, w.f_ext.ravel(), w.pinned)
    np.testing.assert_array_equal(b.positions_get(), d.positions_get())


@pytest.mark.parametrize("dims,radius", [((3, 3, 7), 1.5), ((6, 6, 12), 3.0), ((8, 8, 12), 3.0)],
                         ids=["ragged-tile", "large-unions", "wide-radius"])
def test_mixed_nonlocal_tiles(dims, radius):
    """The tiled Eq. 20 kernel (a tile of tets per CTA, neighbour union staged in
    shared memory) on a mesh whose last tile is partial (378 tets), on one whose
    tile unions exceed 1,792 rows (R_d = 3 on 2,592 tets), and on one whose
    128-tet unions are too wide for four CTAs per SM (R_d = 3 on 4,608 tets), so
    the mesh takes 64-tet tiles; against the oracle.  A single-mesh launch
    stages the mesh's largest union; a batched launch stages 1,792 rows, so in a
    batch the large tiles read global memory: the batch member must give the
    single-mesh drivers bit for bit."""
    from oracle import mesh as omesh
    from workloads import Workload
    from workloads.meshes import jitter, kuhn_box
    nodes, tets, grid = kuhn_box(*dims)
    nodes = jitter(nodes, 0.01, 1.0, 5)
    top = np.nonzero(grid[:, 2] == dims[2])[0]
    f = np.zeros_like(nodes)
    f[top, 0] = 50.0 / len(top)
    pinned = np.nonzero(grid[:, 2] == 0)[0].astype(np.int32)
    w = Workload("box_tiles", nodes, tets, 1e6, 0.3, 1000.0, 1e-3, 3, math.inf, radius, f, pinned)
    T = len(tets)
    nb = omesh.nonlocal_neighbours(nodes, tets, radius)
    unions = [len(set().union(*[set(x) for x in nb[g:g + 128]])) for g in range(0, T, 128)]
    if radius == 1.5:
        assert T % 128 != 0
    else:
        assert max(unions) > 1792   # these tiles take the global-memory path
    # the tile rule: 64 tets where four CTAs with the largest 128-tet union
    # (24 B a row) would not fit 227 KB of shared memory
    tile = 64 if max(unions) * 24 * 4 > 227 * 1024 else 128
    assert tile == (64 if dims == (8, 8, 12) else 128)
    model0 = oracle_model(w, threshold=math.inf, radius=radius)
    st = deformed_state(w, seed=31)
    d0, _, _, _ = model0.damage_update(st)
    theta = float(np.quantile(d0, 0.95))
    model = oracle_model(w, threshold=theta, radius=radius)
    m = mixed_mesh(w, gpu_material(gf, w, threshold=theta, radius=radius))
    assert m.info["eq20_tile"] == tile
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
    s = m.step(w.dt, w.f_ext.ravel(), w.pinned)
    assert s["status"] == 0
    new, info = model.step(st, w.dt, w.f_ext, w.pinned)
    drv, lab = m.damage_get()
    assert_close(drv, info["driver"], rtol=RTOL32, floor=FLOOR32, what="driver (mixed, tiles)")
    assert_labels(lab, info["labels"], info["driver"], theta, band=BAND32)
    assert lab.sum() > 0
    member = mixed_mesh(w, gpu_material(gf, w, threshold=theta, radius=radius))
    member.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
    b = gf.Batch([member])
    sb = b.step(w.dt, [w.f_ext.ravel()], [w.pinned])
    assert sb[0]["status"] == 0
    np.testing.assert_array_equal(member.damage_get()[0], drv)
    b.close()

"""GPU split visualisation mesh (Sec. 4.1) against the oracle, through the C
ABI.  The output is a pure function of the current positions and break
labels, so the oracle is fed the GPU's own state.

Bar: child positions to 1e-13 of the coordinate scale (the same sums in the
same order; any difference is rounding), quads identical (integer work).
"""
import ctypes
import math

import numpy as np
import pytest

from helpers import deformed_state, gpu_material, oracle_model
from oracle import mesh, surface
from workloads import LOAF_AXES, beam_config, loaf_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def test_fractured_beam_surface_matches_oracle():
    w = beam_config()
    st = deformed_state(w, seed=41, amp=0.08)
    model0 = oracle_model(w, threshold=math.inf)
    drv, *_ = model0.damage_update(st)
    theta = float(np.quantile(drv, 0.9))
    m = gf.mesh_create(w.nodes, w.tets, gpu_material(gf, w, threshold=theta))
    m.state_set(x=st.x.ravel(), v=st.v.ravel())
    for _ in range(2):
        m.step(w.dt, w.f_ext.ravel(), w.pinned)
    out = m.surface_get()
    x = m.positions_get().reshape(-1, 3)
    _, lab = m.damage_get()
    assert lab.sum() > 0
    edges, _ = mesh.edges_of(w.tets)
    V, Q, faces, _ = surface.surface(w.nodes, x, w.tets, edges, lab)
    assert out["n_faces"] == len(faces)
    scale = np.abs(V).max()
    np.testing.assert_allclose(out["vertices"], V, rtol=0, atol=1e-13 * scale)
    np.testing.assert_array_equal(out["quads"], Q)


def test_surface_device_output_and_small_capacity():
    w = beam_config()
    m = gf.mesh_create(w.nodes, w.tets, gpu_material(gf, w))
    edges, _ = mesh.edges_of(w.tets)
    rng = np.random.default_rng(5)
    lab = (rng.random(len(edges)) < 0.1).astype(np.uint8)
    x = w.nodes + 0.01 * rng.normal(size=w.nodes.shape)
    m.state_set(x=x.ravel(), v=np.zeros(x.size), labels=lab)
    sz = m.surface_sizes()
    V, Q, _, _ = surface.surface(w.nodes, x, w.tets, edges, lab)
    assert sz["n_quads"] == len(Q) > 0
    lib = gf.load_library()
    Vd = torch.empty((sz["n_vertices"], 3), dtype=torch.float64, device="cuda")
    Qd = torch.empty((sz["n_quads"], 4), dtype=torch.int32, device="cuda")
    nq = ctypes.c_int64()
    assert lib.gf_surface_get(m._h, Vd.data_ptr(), Qd.data_ptr(), sz["n_quads"], gf.MEM_DEVICE, ctypes.byref(nq)) == 0
    np.testing.assert_allclose(Vd.cpu().numpy(), V, rtol=0, atol=1e-13 * np.abs(V).max())
    np.testing.assert_array_equal(Qd.cpu().numpy(), Q)
    assert lib.gf_surface_get(m._h, Vd.data_ptr(), Qd.data_ptr(), sz["n_quads"] - 1, gf.MEM_DEVICE,
                              ctypes.byref(nq)) != 0
    assert nq.value == sz["n_quads"]


def test_loaf_surface_sampled():
    """Half-size loaf with 2% of the edges broken: sampled edges, faces and tets
    against the oracle's rule, and the quad count."""
    w = loaf_config(axes=tuple(0.5 * a for a in LOAF_AXES))
    m = gf.mesh_create(w.nodes, w.tets, gf.material(w.young, w.poisson, w.density))
    edges = m.edges_get().astype(np.int64)
    rng = np.random.default_rng(6)
    lab = (rng.random(len(edges)) < 0.02).astype(np.uint8)
    x = w.nodes + 0.02 * rng.normal(size=w.nodes.shape)
    m.state_set(x=x.ravel(), v=np.zeros(x.size), labels=lab)
    out = m.surface_get()
    V = out["vertices"]
    N, NE = len(w.nodes), len(edges)
    faces, tet_faces = surface.faces_of(w.tets)
    assert out["n_faces"] == len(faces)
    _, tet_edges = mesh.edges_of(w.tets)
    assert len(out["quads"]) == 2 * int(lab[tet_edges].sum())
    eid = {(int(a), int(b)): k for k, (a, b) in enumerate(edges)}

    def broken(u, v):
        return bool(lab[eid[(min(u, v), max(u, v))]])

    for e in rng.choice(NE, 200, replace=False):
        want = surface._follow(w.nodes, x, tuple(int(v) for v in edges[e]), broken)
        np.testing.assert_allclose(V[N + 2 * e:N + 2 * e + 2], want, rtol=0, atol=1e-12)
    for f in rng.choice(len(faces), 200, replace=False):
        want = surface._follow(w.nodes, x, tuple(int(v) for v in faces[f]), broken)
        o = N + 2 * NE + 3 * f
        np.testing.assert_allclose(V[o:o + 3], want, rtol=0, atol=1e-12)
    o2 = N + 2 * NE + 3 * len(faces)
    for t in rng.choice(len(w.tets), 200, replace=False):
        want = surface._follow(w.nodes, x, tuple(int(v) for v in w.tets[t]), broken)
        np.testing.assert_allclose(V[o2 + 4 * t:o2 + 4 * t + 4], want, rtol=0, atol=1e-12)

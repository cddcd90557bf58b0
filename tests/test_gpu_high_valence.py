"""GPU parity on a mesh of high-valence nodes: 400 disjoint fans, each a hub
node and two apexes joined to a ring of 40 nodes, so the hub and apex block
rows hold 42-43 blocks (more than the 16 lanes of a half-warp takes at once,
and unequal lengths in the two rows a half-warp of the inner SpMV carries at a
time; the loaf's rows hold at most 15).  One step from a deformed state in every
solver-loop form, against the oracle: FP64 forms at the FP64 bar, mixed forms
at the reduced-precision bar.
"""
import numpy as np
import pytest

from helpers import assert_norm_close, deformed_state, gpu_material, oracle_model
from workloads import Workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

M, K = 40, 400   # ring nodes per fan, fans


def fans():
    a = 2 * np.pi * np.arange(M) / M
    ring = np.stack([np.cos(a), np.sin(a), np.zeros(M)], 1)
    one = np.concatenate([[[0.0, 0.0, 0.0]], ring, [[0.0, 0.0, 0.8]], [[0.0, 0.0, -0.8]]])
    hub, top, bot = 0, M + 1, M + 2
    tets = []
    for i in range(M):
        r0, r1 = 1 + i, 1 + (i + 1) % M
        tets += [[hub, r0, r1, top], [hub, r1, r0, bot]]
    tets = np.array(tets)
    P = one[tets]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    tets[vol < 0] = tets[vol < 0][:, [0, 2, 1, 3]]
    n1 = len(one)
    nodes = np.concatenate([one + np.array([3.0 * (k % 20), 3.0 * (k // 20), 0.0]) for k in range(K)])
    tets = np.concatenate([tets + k * n1 for k in range(K)]).astype(np.int32)
    f = np.zeros_like(nodes)
    f[top::n1, 2] = 50.0
    return Workload("fans_400x40", nodes, tets, 1e5, 0.3, 1000.0, 1e-3, 1, np.inf, 0.5, f, np.zeros(0, np.int32))


@pytest.fixture(scope="module")
def case():
    w = fans()
    st = deformed_state(w, seed=41, amp=0.02, vamp=0.05)
    new, _ = oracle_model(w).step(st, w.dt, w.f_ext, w.pinned)
    return w, st, new


@pytest.mark.parametrize("precision,solve,rtol", [
    (gf.FP64, gf.SOLVE_KERNELS, 1e-9), (gf.FP64, gf.SOLVE_CG, 1e-9), (gf.FP64, gf.SOLVE_NESTED, 1e-9),
    (gf.MIXED, gf.SOLVE_CG, 1e-5), (gf.MIXED, gf.SOLVE_KERNELS, 1e-5), (gf.MIXED, gf.SOLVE_PERSISTENT, 1e-5)])
def test_high_valence_rows_step_matches_oracle(case, precision, solve, rtol):
    w, st, new = case
    m = gf.mesh_create(w.nodes, w.tets, gpu_material(gf, w), precision=precision, cg_rtol=1e-12, cg_maxit=20000)
    m.tuning_set(solve_loop=solve)
    m.state_set(x=st.x.ravel(), v=st.v.ravel())
    s = m.step(w.dt, w.f_ext.ravel())
    assert s["status"] == 0 and s["rel_res"] <= 1e-12 and s["cg_iters"] > 0
    assert_norm_close(m.velocities_get(), new.v, rtol=rtol, what=f"v ({precision}, form {solve})")
    m.close()

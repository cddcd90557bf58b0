"""GPU test of the allocation-free solve, gf_bsr_pcg_solve_static.

That entry point is for callers that cannot allocate device memory while they
solve (device-wide synchronisation of cudaMalloc/cudaFree, or a memory budget
fixed up front): its scratch lives in a fixed array inside the library.  Here it
solves, through the C ABI, the very systems that gf_step assembled and solved,
twice in a row (the shared scratch keeps the first call's contents), and its
solutions must match gf_step's velocity updates within the FP64 parity bound of
the other GPU tests.  The free rows of x are never read: the second call passes
NaN there.  A free row without a diagonal block is refused.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from helpers import RTOL64, assert_norm_close, deformed_state
from workloads import beam_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def test_static_solve_matches_step_solver_two_calls():
    w = beam_config()
    mat = gf.material(w.young, w.poisson, w.density, threshold=float("inf"), radius=w.radius, beta=1e-3)
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-13, cg_maxit=20000)
    fixed = np.zeros(w.n_nodes, np.uint8)
    fixed[w.pinned] = 1
    for call, seed in enumerate((4, 9)):
        st = deformed_state(w, seed=seed, amp=0.02, vamp=0.1)
        m.state_set(x=st.x.ravel(), v=st.v.ravel())
        stats = m.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert stats["status"] == 0
        rp, col, val, rhs = m.system_get()
        dv = m.velocities_get() - st.v.ravel()
        x0 = np.full(3 * w.n_nodes, 0.0 if call == 0 else np.nan)
        x0.reshape(-1, 3)[w.pinned] = dv.reshape(-1, 3)[w.pinned]      # prescribed rows (-v_old)
        dev = dict(device="cuda")
        x = torch.tensor(x0, dtype=torch.float64, **dev)
        iters, rel = gf.bsr_pcg_solve_static(
            torch.tensor(rp, **dev), torch.tensor(col, **dev), torch.tensor(val.ravel(), **dev),
            torch.tensor(rhs, **dev), x, torch.tensor(fixed, **dev), rtol=1e-13, maxit=20000)
        assert iters > 0 and rel <= 1e-12, (call, iters, rel)
        assert_norm_close(x.cpu().numpy(), dv, rtol=RTOL64, what=f"static solve, call {call}")


def test_static_solve_rejects_oversized_systems():
    n = 32769
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    vals = torch.zeros(9, dtype=torch.float64, device="cuda")
    b = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    x = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GraphFEMError) as e:
        gf.bsr_pcg_solve_static(rp, col, vals, b, x)
    assert e.value.status == 1 and "32768" in str(e.value)


def test_static_solve_refuses_a_free_row_without_diagonal_block():
    # two block rows: row 0 holds its diagonal block, row 1 only the (1, 0) block
    dev = dict(device="cuda")
    rp = torch.tensor([0, 1, 2], dtype=torch.int32, **dev)
    col = torch.tensor([0, 0], dtype=torch.int32, **dev)
    vals = torch.tensor(np.concatenate([np.eye(3).ravel(), 0.5 * np.eye(3).ravel()]), dtype=torch.float64, **dev)
    b = torch.ones(6, dtype=torch.float64, **dev)
    x = torch.zeros(6, dtype=torch.float64, **dev)
    with pytest.raises(gf.GraphFEMError) as e:
        gf.bsr_pcg_solve_static(rp, col, vals, b, x)
    assert e.value.status == 1 and "diagonal" in str(e.value)
    # the same system with row 1 held fixed solves (row 0 alone: x0 = b0 - 0)
    fixed = torch.tensor([0, 1], dtype=torch.uint8, **dev)
    iters, rel = gf.bsr_pcg_solve_static(rp, col, vals, b, x, fixed, rtol=1e-12)
    assert rel <= 1e-12
    np.testing.assert_allclose(x.cpu().numpy(), [1, 1, 1, 0, 0, 0], rtol=1e-14)

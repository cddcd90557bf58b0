"""GPU parity of the quasi-static load step (Eq. 36; Newton with an energy line
search, Sec. 4.3) against the oracle, through the C ABI.

The converged equilibrium is what is unique (the two sides may take
different step lengths on the way), so it is what is compared: positions
within 1e-9 of each node's displacement plus 1e-10 of the largest (the
oracle's residual floor is ~1e-10 of the first residual), drivers to 1e-9,
labels equal outside the threshold band, from identical start states.  Both
linear solvers of the Newton iterations are held to this bar: the FP64 PCG and
the flexible FP64 PCG preconditioned by an inner FP32 PCG (it stops at the same
FP64 residual test, so the Newton iterates solve the same FP64 systems).
"""
import math

import numpy as np
import pytest

from helpers import assert_close, assert_labels, assert_positions_close, oracle_model
from oracle.step import Material, Model
from workloads import kuhn_box

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

E, NU, RHO = 1e6, 0.3, 1000.0


def bar(nz=8):
    X, T, grid = kuhn_box(2, 2, nz)
    lo = np.nonzero(grid[:, 2] == 0)[0]
    hi = np.nonzero(grid[:, 2] == nz)[0]
    return X, T.astype(np.int32), lo, hi


SOLVERS = [gf.QS_SOLVE_FP64, gf.QS_SOLVE_NESTED]


def meshes(X, T, energy, threshold, radius=1.5, solver=gf.QS_SOLVE_FP64):
    model = Model(X, T, Material(E, NU, RHO, threshold=threshold, radius=radius, energy=energy))
    mat = gf.material(E, NU, RHO, threshold=threshold, radius=radius,
                      energy=gf.ENERGY_SNH if energy == "snh" else gf.ENERGY_STVK)
    m = gf.mesh_create(X, T, mat, cg_rtol=1e-13, cg_maxit=20000)
    m.quasistatic_solver_set(solver)
    return model, m


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("energy", ["stvk", "snh"])
def test_pulled_bar_load_steps_match_oracle(energy, solver):
    """Both ends pinned, one end pulled 4% per load step; the threshold is set
    so that edges break from the second step on.  Each GPU step starts from the
    oracle's state."""
    X, T, lo, hi = bar()
    pins = np.concatenate([lo, hi]).astype(np.int32)
    probe, _ = meshes(X, T, energy, math.inf)
    st = probe.rest_state()
    target = X[pins].copy()
    target[len(lo):, 2] += 0.32
    st1, _ = probe.quasistatic_step(st, np.zeros_like(X), pins, target)
    drv, *_ = probe.damage_update(st1)
    theta = float(np.quantile(drv, 0.97))
    model, m = meshes(X, T, energy, theta, solver=solver)
    st = model.rest_state()
    broke = 0
    for k in range(1, 4):
        target = X[pins].copy()
        target[len(lo):, 2] += 0.32 * k
        m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        stats = m.quasistatic_step(None, pins, target, max_newton=60, rtol=1e-11)
        new, info = model.quasistatic_step(st, np.zeros_like(X), pins, target)
        assert stats["status"] == 0 and stats["rel_res"] <= 1e-11 and stats["newton_iters"] >= 2
        d, lab = m.damage_get()
        assert_close(d, info["driver"], what="driver", floor=0.0, abs_floor=1e-13)
        assert_labels(lab, info["labels"], info["driver"], theta)
        if np.array_equal(lab, info["labels"]):
            assert_positions_close(m.positions_get(), new.x, st.x, what="x", noise=1e-10)
        assert np.abs(m.velocities_get()).max() == 0.0
        broke += int(lab.sum())
        st = new
    assert broke > 0


@pytest.mark.parametrize("solver", SOLVERS)
def test_tip_load_on_a_clamped_bar_matches_oracle(solver):
    X, T, lo, hi = bar(nz=10)
    model, m = meshes(X, T, "stvk", math.inf, solver=solver)
    f = np.zeros_like(X)
    f[hi, 0] = 40.0
    st = model.rest_state()
    stats = m.quasistatic_step(f.ravel(), lo.astype(np.int32), None, max_newton=60, rtol=1e-10)
    new, info = model.quasistatic_step(st, f, lo, None)
    assert stats["status"] == 0 and stats["newton_iters"] >= 3
    assert_positions_close(m.positions_get(), new.x, st.x, what="x", noise=1e-10)


def test_quasistatic_step_is_refused_on_mixed_meshes():
    X, T, lo, hi = bar(nz=4)
    m = gf.mesh_create(X, T, gf.material(E, NU, RHO), precision=gf.MIXED)
    with pytest.raises(gf.GraphFEMError):
        m.quasistatic_step(None, lo.astype(np.int32), None)
    with pytest.raises(gf.GraphFEMError) as e:
        m.quasistatic_solver_set(gf.QS_SOLVE_NESTED)
    assert e.value.status == 8
    m64 = gf.mesh_create(X, T, gf.material(E, NU, RHO))
    for bad in ((2, 1e-3), (gf.QS_SOLVE_NESTED, 1.0), (gf.QS_SOLVE_NESTED, float("nan"))):
        with pytest.raises(gf.GraphFEMError) as e:
            m64.quasistatic_solver_set(*bad)
        assert e.value.status == 1


def test_nested_solve_inner_tolerances():
    """The nested solve on a stiff clamped bar (bending, where the FP32 matrix's
    rounding matters most) at loose to tight inner tolerances: every run meets
    the Newton tolerance and lands on the FP64 solver's equilibrium."""
    X, T, lo, hi = bar(nz=12)
    f = np.zeros_like(X)
    f[hi, 0] = 40.0
    _, ref = meshes(X, T, "stvk", math.inf)
    s_ref = ref.quasistatic_step(f.ravel(), lo.astype(np.int32), None, max_newton=60, rtol=1e-10)
    assert s_ref["status"] == 0
    for tol in (1e-1, 1e-3, 1e-5):
        _, m = meshes(X, T, "stvk", math.inf, solver=gf.QS_SOLVE_NESTED)
        m.quasistatic_solver_set(gf.QS_SOLVE_NESTED, tol)
        s = m.quasistatic_step(f.ravel(), lo.astype(np.int32), None, max_newton=60, rtol=1e-10)
        assert s["status"] == 0 and s["rel_res"] <= 1e-10 and s["cg_iters"] > 0
        assert_positions_close(m.positions_get(), ref.positions_get(), X, what=f"x (inner rtol {tol})", noise=1e-10)
        m.close()


@pytest.mark.parametrize("solver", SOLVERS)
def test_fragmenting_pull_stays_finite(solver):
    """A pull far past the break threshold separates pieces: nodes left without
    stiffness keep their positions and the step returns finite positions
    (no mass regularises the quasi-static system)."""
    X, T, lo, hi = bar(nz=8)
    model, m = meshes(X, T, "stvk", 1e-3, solver=solver)
    pins = np.concatenate([lo, hi]).astype(np.int32)
    for k in range(1, 4):
        target = X[pins].copy()
        target[len(lo):, 2] += 0.4 * k
        s = m.quasistatic_step(None, pins, target, max_newton=30, rtol=1e-8)
        assert s["status"] == 0
    x = m.positions_get().reshape(-1, 3)
    assert np.isfinite(x).all()
    assert (m.chi_get() == 0).sum() > 0
    np.testing.assert_allclose(x[pins], target, rtol=0, atol=1e-12)

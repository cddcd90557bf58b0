"""Full-size parity on the 620k-tet loaf mesh, in the configurations bench.py
times: the ductile loaf in FP64 and mixed precision, and the brittle glass
point impact in mixed precision, CG to 1e-6.  The oracle cannot step the whole
mesh in seconds, so it recomputes sampled outputs one by one: four compact
regions of tets, whose edge drivers and labels (Eq. 20-21), chi (Eq. 25), and
the matrix rows and right-hand sides of their interior nodes (Eq. 2, 12,
32-34) it evaluates from the same start state.  Properties that hold at any size are checked on the
whole mesh: the solver residual recomputed on the host from the GPU's own
system, the position update, and monotone labels."""
import numpy as np
import pytest
import scipy.sparse as sp

from helpers import LABEL_BAND, assert_close, assert_norm_close
from oracle import damage, elastic, mesh as omesh
from workloads import glass_config, loaf_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402


def seeded_state(w, seed, strain, speed, broken):
    """A smooth seeded displacement field of the given strain scale, random
    velocities and a random 0.3% (``broken``) of edges already broken."""
    rng = np.random.default_rng(seed)
    X = w.nodes
    L = X.max(0) - X.min(0)
    u = np.zeros_like(X)
    ph = rng.uniform(0, 2 * np.pi, size=(3, 3))
    for c in range(3):
        for d in range(3):
            u[:, c] += strain * L[d] / 6 * np.sin(2 * np.pi * X[:, d] / L[d] + ph[c, d])
    x = X + u + 0.025 * strain * rng.normal(size=X.shape)
    v = speed * rng.normal(size=X.shape)
    edges, tet_edges = omesh.edges_of(w.tets)
    labels0 = (rng.uniform(size=len(edges)) < broken).astype(np.uint8)
    return x, v, edges, tet_edges, labels0


@pytest.fixture(scope="module")
def loaf():
    w = loaf_config()
    return (w,) + seeded_state(w, 21, 0.004, 0.01, 0.003)


@pytest.fixture(scope="module")
def glass():
    """The brittle glass configuration: the loaf mesh, E = 7e10, nu = 0.22,
    rho = 2500, the lowest 5% of nodes pinned and a 1e4 N point impact at the
    top apex; a state at glass-like strains (1e-5)."""
    w = glass_config()
    return (w,) + seeded_state(w, 23, 1e-5, 1e-4, 0.003)


def oracle_region_state(w, x, labels, edges, tet_edges, centres, lam, mu, radius):
    """Oracle quantities around the sample regions (global tet / edge ids)."""
    X, tets = w.nodes, w.tets.astype(np.int64)
    cen = omesh.centroids(X, tets)
    V_all, _, _ = omesh.rest_geometry(X, tets)
    d_reg = np.min(np.linalg.norm(cen[:, None, :] - centres[None], axis=2), axis=1)
    T_s = np.nonzero(d_reg <= 2.5)[0]                                  # sampled tets
    E_s = np.unique(tet_edges[T_s])                                    # their edges
    # tets incident to the sampled edges (their sigma-bar enters the edge driver)
    inc = np.nonzero(np.isin(tet_edges, E_s).any(1))[0]
    # stresses and chi_old are needed for every neighbour of those tets
    need = np.nonzero(d_reg <= 2.5 + 2.0 + radius)[0]
    V, D2, q = omesh.rest_geometry(X, tets[need])
    s = elastic.squared_edge_lengths(x, tets[need])
    C = elastic.cauchy_green_lsq(s, D2, q)
    S = damage.stress_voigt(C, lam, mu)
    T = damage.projection_T(x, tets[need], 2.0)
    sigf = np.einsum("tkc,tc->tk", T, S)
    chi_old = damage.chi(labels, tet_edges[need], sigf, w.young)
    sig_in = np.full((len(tets), 6), np.nan)
    sig_in[need] = S * chi_old[:, None]
    nb = omesh.nonlocal_neighbours(X, tets, radius, subset=inc)
    wts = damage.nonlocal_weights(cen, V_all, nb, radius, subset=inc)
    sig_bar = damage.nonlocal_average(sig_in, nb, wts)
    assert np.isfinite(sig_bar).all()
    T_inc = damage.projection_T(x, tets[inc], 2.0)
    sig_star = np.einsum("tkc,tc->tk", T_inc, sig_bar)
    drv = np.full(len(edges), -np.inf)
    np.maximum.at(drv, tet_edges[inc].ravel(), sig_star.ravel())
    drv /= w.young
    pos = {t: i for i, t in enumerate(need)}
    return dict(T_s=T_s, E_s=E_s, driver=drv, need=need, pos=pos, sigf=sigf)


# per precision: element-wise rtol, floor (of the sampled array's scale), label band
TOL = {"fp64": dict(rtol=1e-9, floor_drv=0.0, abs_drv=1e-13, floor_chi=1e-12, floor_A=1e-12, floor_b=1e-9,
                    band=LABEL_BAND),
       "mixed": dict(rtol=1e-5, floor_drv=1e-6, abs_drv=0.0, floor_chi=1e-6, band=1e-5, floor_row=1e-5)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_loaf_fullsize_sampled_parity(loaf, precision):
    """Both forms bench.py times, on the full loaf.  FP64: element-wise 1e-9.
    Mixed: the FP32 tolerance 1e-5 (label band 1e-5); the sampled matrix rows
    and rhs norm-wise at 1e-5 and element-wise at 1e-5 of each entry plus 1e-5
    of the row's largest entry (matrix) or of the largest sampled entry (rhs):
    FP32 strains from displacement differences carry ~1e-6 relative error, and
    the edge-space sums forming a nodal force amplify it about tenfold on single
    entries that cancel (a rhs entry misses 1e-5 of its own three-entry row by
    up to 1.5x)."""
    sampled_parity(loaf, precision)


def test_glass_fullsize_sampled_parity(glass):
    """The glass point impact in mixed precision on the full mesh, at the 1e-5
    bar of reduced precision: sampled drivers, labels, chi, matrix rows and
    rhs against the oracle, and the FP64-accurate solve residual over the free
    DOFs with the bottom nodes pinned."""
    w = glass[0]
    stats = sampled_parity(glass, "mixed", pinned=w.pinned)
    assert stats["cg_iters"] > 2 * stats["refine_sweeps"]     # the stiff case: many inner iterations


def threshold_in_gap(drv, q):
    """A threshold near the q-quantile of the sampled drivers, at the middle of
    the widest relative gap among the 41 sorted drivers around it, so that no
    sampled driver lies within the label band of it and the labels, chi and
    system of the sampled tets must agree exactly."""
    d = np.sort(drv[np.isfinite(drv)])
    k = int(q * (len(d) - 1))
    lo, hi = max(k - 20, 0), min(k + 20, len(d) - 1)
    gaps = (d[lo + 1:hi + 1] - d[lo:hi]) / np.abs(d[lo + 1:hi + 1])
    i = lo + int(np.argmax(gaps))
    return float(0.5 * (d[i] + d[i + 1]))


def sampled_parity(case, precision, pinned=None):
    tol = TOL[precision]
    w, x, v, edges, tet_edges, labels0 = case
    lam, mu = elastic.lame(w.young, w.poisson)
    rng = np.random.default_rng(7)
    centres = w.nodes[rng.choice(w.n_nodes, 4, replace=False)]
    reg = oracle_region_state(w, x, labels0, edges, tet_edges, centres, lam, mu, w.radius)
    E_s, T_s = reg["E_s"], reg["T_s"]
    theta = threshold_in_gap(reg["driver"][E_s], 0.9)
    m = gf.mesh_create(w.nodes, w.tets, gf.material(w.young, w.poisson, w.density, threshold=theta,
                                                    radius=w.radius), cg_rtol=1e-6,
                       precision=gf.MIXED if precision == "mixed" else gf.FP64)
    np.testing.assert_array_equal(m.edges_get(), edges)
    m.state_set(x=x.ravel(), v=v.ravel(), labels=labels0)
    f = w.f_ext
    stats = m.step(w.dt, f.ravel(), pinned)
    assert stats["status"] == 0
    drv, lab = m.damage_get()
    # (1) drivers and labels of the sampled edges
    assert_close(drv[E_s], reg["driver"][E_s], rtol=tol["rtol"], floor=tol["floor_drv"], abs_floor=tol["abs_drv"],
                 what="driver")
    want_lab = labels0 | (reg["driver"] >= theta)
    diff = E_s[lab[E_s] != want_lab[E_s]]
    assert np.all(np.abs(reg["driver"][diff] - theta) <= tol["band"] * theta)
    assert lab[E_s].sum() > 0
    # labels never heal anywhere
    assert np.all(lab >= labels0)
    # (2) chi of the sampled tets from the new labels of their edges
    new_lab = labels0.copy()
    new_lab[E_s] = want_lab[E_s]
    sigf_s = reg["sigf"][[reg["pos"][t] for t in T_s]]
    chi_s = damage.chi(new_lab, tet_edges[T_s], sigf_s, w.young)
    chi_gpu = m.chi_get()
    # labels inside the band may differ; chi and the system then differ too, so
    # those checks need identical labels on the sample (they are, at these seeds)
    assert np.array_equal(lab[E_s], new_lab[E_s])
    assert_close(chi_gpu[T_s], chi_s, rtol=tol["rtol"], floor=tol["floor_chi"], what="chi")
    assert (chi_s < 1).any()
    # (3) matrix rows and rhs of nodes whose incident tets all lie in T_s
    tets = w.tets.astype(np.int64)
    in_s = np.zeros(w.n_tets, bool)
    in_s[T_s] = True
    node_all_in = np.ones(w.n_nodes, bool)
    np.logical_and.at(node_all_in, tets.ravel(), np.repeat(in_s, 4))
    free = np.ones(w.n_nodes, bool)
    if pinned is not None:
        free[pinned] = False
    N_s = np.nonzero(node_all_in & free & np.isin(np.arange(w.n_nodes), tets[T_s].ravel()))[0]
    assert len(N_s) >= 4
    V, D2, q = omesh.rest_geometry(w.nodes, tets[T_s])
    Ke = elastic.element_tangent(x, tets[T_s], V, D2, q, lam, mu, chi_s)
    fe = elastic.element_forces(x, tets[T_s], V, D2, q, lam, mu, chi_s)
    mass = omesh.lumped_mass(w.nodes, tets, w.density, omesh.rest_geometry(w.nodes, tets)[0])
    dt = w.dt
    rp, col, val, rhs = m.system_get()
    got_b, want_bs = [], []
    for n in N_s:
        want_row = {}
        want_b = dt * (f[n] - 0.0 * v[n])
        for e_i, t in enumerate(T_s):
            loc = np.nonzero(tets[t] == n)[0]
            if not len(loc):
                continue
            a = loc[0]
            ve = v[tets[t]].ravel()
            Kv = Ke[e_i] @ ve
            want_b = want_b + dt * (fe[e_i, a] - dt * Kv[3 * a:3 * a + 3])
            for b in range(4):
                blk = dt * dt * Ke[e_i][3 * a:3 * a + 3, 3 * b:3 * b + 3]
                want_row[tets[t, b]] = want_row.get(tets[t, b], 0.0) + blk
        want_row[n] = want_row[n] + mass[n] * np.eye(3)
        cols = col[rp[n]:rp[n + 1]]
        assert sorted(want_row) == list(cols)
        got = val[rp[n]:rp[n + 1]]
        want = np.stack([want_row[c] for c in cols])
        if precision == "fp64":
            assert_close(got, want, rtol=tol["rtol"], floor=tol["floor_A"], what=f"A row {n}")
        else:
            assert_norm_close(got, want, rtol=tol["rtol"], what=f"A row {n} (mixed)")
            # element-wise too, against the row's largest entry: entries that
            # cancel to near zero carry the FP32 rounding of the whole row
            assert_close(got, want, rtol=tol["rtol"], floor=tol["floor_row"], what=f"A row {n} (mixed, element-wise)")
        got_b.append(rhs[3 * n:3 * n + 3])
        want_bs.append(want_b)
    if precision == "fp64":
        assert_close(np.array(got_b), np.array(want_bs), rtol=tol["rtol"], floor=tol["floor_b"], what="rhs rows")
    else:
        assert_norm_close(np.array(got_b), np.array(want_bs), rtol=tol["rtol"], what="rhs rows (mixed)")
        # element-wise against the largest sampled entry: a nodal force is a sum
        # of element forces that cancel, each carrying FP32 rounding
        assert_close(np.array(got_b), np.array(want_bs), rtol=tol["rtol"], floor=tol["floor_row"],
                     what="rhs rows (mixed, element-wise)")
    # (4) the solve: residual over the free DOFs recomputed on the host from the
    # GPU's own system, relative to b_free = b - A_fp dv_p (prescribed rows)
    rows = np.repeat(np.arange(w.n_nodes), np.diff(rp))
    r3 = (3 * rows[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
    c3 = (3 * col[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
    A = sp.csr_matrix((val.ravel(), (r3.ravel(), c3.ravel())), shape=(3 * w.n_nodes, 3 * w.n_nodes))
    v_new = m.velocities_get()
    dv = v_new - v.ravel()
    fr = np.repeat(free, 3)
    # prescribed: at rest (the mixed path carries dv as a float pair: zero to its rounding)
    assert np.abs(v_new.reshape(-1, 3)[~free]).max(initial=0.0) <= 1e-12 * np.abs(v).max()
    dvp = np.where(fr, 0.0, dv)
    res = np.linalg.norm((rhs - A @ dv)[fr]) / np.linalg.norm((rhs - A @ dvp)[fr])
    assert res <= 1e-6
    assert abs(res - stats["rel_res"]) <= 1e-3 * res + 1e-15
    # (5) position update x_new = x + dt v_new
    np.testing.assert_allclose(m.positions_get(), x.ravel() + dt * v_new, rtol=1e-15, atol=1e-15)
    m.close()
    return stats


def test_loaf_quasistatic_nested_solve_matches_fp64_solver():
    """One quasi-static load step of the full loaf (end caps pulled apart by
    1e-4 of the length, Newton to 1e-6) with each linear solver of the Newton
    iterations: the nested solve (flexible FP64 PCG, FP32 inner PCG) stops at
    the FP64 PCG's residual test, so both reach the same equilibrium: the same
    labels and Newton iteration count, positions within 1e-7 of the largest
    displacement (each Newton system is solved to cg_rtol 1e-6, so the two
    iterates differ by the solver error, far below the load step)."""
    w = loaf_config()
    X = w.nodes
    L = X[:, 0].max() - X[:, 0].min()
    lo = np.nonzero(X[:, 0] <= X[:, 0].min() + 0.1 * L)[0].astype(np.int32)
    hi = np.nonzero(X[:, 0] >= X[:, 0].max() - 0.1 * L)[0].astype(np.int32)
    pins = np.concatenate([lo, hi])
    target = X[pins].copy()
    target[:len(lo), 0] -= 1e-4 * L
    target[len(lo):, 0] += 1e-4 * L
    mat = gf.material(w.young, w.poisson, w.density, threshold=w.threshold, radius=w.radius)
    out = {}
    for solver in (gf.QS_SOLVE_FP64, gf.QS_SOLVE_NESTED):
        m = gf.mesh_create(X, w.tets, mat, cg_rtol=w.cg_rtol)
        m.quasistatic_solver_set(solver)
        s = m.quasistatic_step(None, pins, target, max_newton=20, rtol=1e-6)
        assert s["status"] == 0 and s["rel_res"] <= 1e-6 and s["cg_iters"] > 0
        out[solver] = (s, m.positions_get(), m.damage_get()[1])
        m.close()
    (s64, x64, l64), (sn, xn, ln) = out[gf.QS_SOLVE_FP64], out[gf.QS_SOLVE_NESTED]
    assert sn["newton_iters"] == s64["newton_iters"]
    np.testing.assert_array_equal(ln, l64)
    d = np.abs(x64 - X.ravel()).max()
    assert d > 0 and np.abs(xn - x64).max() <= 1e-7 * d
    np.testing.assert_allclose(xn.reshape(-1, 3)[pins], target, rtol=0, atol=1e-12)

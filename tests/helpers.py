"""Shared helpers of the GPU parity tests (oracle set-up, states, tolerances)."""
import numpy as np

from oracle.step import Material as OMaterial
from oracle.step import Model, State

# FP64 parity tolerance: relative, element by element with an absolute floor
# tied to the array's scale (entries formed by cancellation).
RTOL64 = 1e-9
# label band: edges whose driver lies within 1e-6 relative of the threshold may differ
LABEL_BAND = 1e-6


def oracle_model(w, threshold=None, radius=None, **kw):
    mat = OMaterial(w.young, w.poisson, w.density,
                    threshold=w.threshold if threshold is None else threshold,
                    radius=w.radius if radius is None else radius, **kw)
    return Model(w.nodes, w.tets, mat)


def gpu_material(gf, w, threshold=None, radius=None, alpha=0.0, beta=0.0, driver_mode="strain",
                 shear_coef=2.0, average_degraded=True):
    return gf.material(w.young, w.poisson, w.density,
                       threshold=w.threshold if threshold is None else threshold,
                       radius=w.radius if radius is None else radius, alpha=alpha, beta=beta,
                       driver_mode=0 if driver_mode == "strain" else 1, shear_coef=int(shear_coef),
                       average_degraded=average_degraded)


def deformed_state(w, seed=0, amp=0.05, vamp=0.2) -> State:
    """A smooth large deformation (strains of a few percent) plus noise and a
    random velocity field: exercises stress, damage and the tangent."""
    rng = np.random.default_rng(seed)
    X = w.nodes
    L = X.max(0) - X.min(0)
    ph = rng.uniform(0, 2 * np.pi, size=(3, 3))
    u = np.zeros_like(X)
    for c in range(3):
        for d in range(3):
            u[:, c] += amp * L[d] / 6 * np.sin(2 * np.pi * X[:, d] / L[d] + ph[c, d])
    u += 0.002 * rng.normal(size=X.shape)
    v = vamp * rng.normal(size=X.shape)
    ne = len(np.unique(np.sort(w.tets[:, [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]]].reshape(-1, 2), 1), axis=0))
    return State(X + u, v, np.zeros(ne, np.uint8), np.ones(w.n_tets))


def assert_close(got, want, rtol=RTOL64, floor=1e-12, what="", abs_floor=0.0):
    """|got - want| <= rtol |want| + floor * max|want| + abs_floor, element-wise."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want)
    bad = err > rtol * np.abs(want) + floor * scale + abs_floor
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} entries differ; worst abs {err.max():.3e} "
                           f"(scale {scale:.3e}) at {np.argmax(err)}")


def assert_norm_close(got, want, rtol=RTOL64, what=""):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    den = np.linalg.norm(want)
    err = np.linalg.norm(got - want)
    assert err <= rtol * den, f"{what}: ||diff|| / ||ref|| = {err / den:.3e} > {rtol}"


def assert_labels(got, want, driver_ref, threshold, band=LABEL_BAND, what="labels"):
    diff = np.nonzero(np.asarray(got) != np.asarray(want))[0]
    if len(diff):
        near = np.abs(driver_ref[diff] - threshold) <= band * abs(threshold)
        assert near.all(), f"{what}: {int((~near).sum())} labels differ outside the threshold band"


def block_values_from_csr(A, row_ptr, col):
    """Values of the scalar CSR matrix A at the 3x3 blocks of a block-CSR pattern."""
    A = A.tocsr()
    nb = len(col)
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    out = np.zeros((nb, 3, 3))
    for a in range(3):
        for b in range(3):
            out[:, a, b] = np.asarray(A[3 * rows + a, 3 * col + b]).ravel()
    return out


def assert_positions_close(got, want, start, rtol=RTOL64, ulps=4.0, what="x", noise=1e-10):
    """Positions after a step: |got - want| <= rtol |dx| + noise max|dx| + ulps eps |want|.
    The ulp term covers the rounding of x + dt v itself (x ~ 10 m, dx ~ 1e-6 m); the
    noise term covers nodes the load has not reached yet, whose displacement (1e-17 m
    after one step) is the rounding noise of the rest-state forces on either side."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    start = np.asarray(start, np.float64).ravel()
    err = np.abs(got - want)
    dx = np.abs(want - start)
    bound = rtol * dx + noise * dx.max() + ulps * np.finfo(np.float64).eps * np.abs(want)
    bad = err > bound
    idx = np.nonzero(bad)[0][:6]
    assert not bad.any(), (f"{what}: {bad.sum()} entries beyond rtol*|dx| + {ulps} ulp; worst {err.max():.3e}; "
                           f"first: idx {idx.tolist()} got {got[idx].tolist()} want {want[idx].tolist()} "
                           f"start {start[idx].tolist()}")

"""Synthetic tetrahedral meshes and load cases.

The paper's own meshes (a loaf from free3d.com, Stanford models, a femur;
Sec. 4.3) are not available, so these seeded generators stand in for them:

* ``kuhn_box``      — a box of unit cubes, each split into the 6 Kuhn tets
                      (one per permutation of the three axis steps); the
                      three-point-bending beam and the batched boxes.
* ``bcc_ellipsoid`` — the body-centred-cubic tetrahedral lattice (cube
                      corners + cube centres; each tet joins two face-adjacent
                      centres to one edge of their shared face) clipped by an
                      ellipsoid on tet centroids; the 620k-tet loaf stand-in
                      of Table 2's "Loaf" row.
* ``two_tet_fig4``  — the two tets sharing a face of Fig. 4.

Everything here is geometry, index selection and random numbers; none of the
method's arithmetic lives in this module.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """A mesh plus its material, loads and constraints (one benchmark case)."""
    name: str
    nodes: np.ndarray          # (n, 3) float64 rest positions
    tets: np.ndarray           # (t, 4) int32
    young: float
    poisson: float
    density: float
    dt: float
    steps: int
    threshold: float           # driver threshold (dimensionless strain units)
    radius: float              # non-local support R_d
    f_ext: np.ndarray          # (n, 3) float64 external nodal forces
    pinned: np.ndarray         # (p,) int32 pinned node ids
    alpha: float = 0.0
    beta: float = 0.0
    cg_rtol: float = 1e-6
    precision: str = "fp64"
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


# --------------------------------------------------------------------------
# lattices
# --------------------------------------------------------------------------

def kuhn_box(nx: int, ny: int, nz: int, h: float = 1.0):
    """Grid [0,nx]x[0,ny]x[0,nz] (spacing h), each cube split into 6 Kuhn tets.

    Node id of lattice point (i, j, k) is ``(i*(ny+1) + j)*(nz+1) + k``.
    Returns (nodes float64 (n,3), tets int32 (6*nx*ny*nz, 4), grid index (n,3)).
    """
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    grid = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], 1).astype(np.int64)
    nodes = grid.astype(np.float64) * h

    def nid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros((4, 3), np.int64)
        for s, ax in enumerate(perm):
            p[s + 1] = p[s]
            p[s + 1, ax] += 1
        tets.append(np.stack([nid(ci + p[v, 0], cj + p[v, 1], ck + p[v, 2]) for v in range(4)], 1))
    # interleave so the 6 tets of a cube are adjacent (spatially coherent order)
    tets = np.stack(tets, 1).reshape(-1, 4).astype(np.int32)
    return nodes, tets, grid


def bcc_ellipsoid(a: float, b: float, c: float, h: float = 1.0):
    """BCC tetrahedral lattice clipped by (x/a)^2+(y/b)^2+(z/c)^2 <= 1 on tet centroids.

    Cube corners sit on integer lattice points, cube centres at half-integers
    (units of h); the ellipsoid is centred at the origin.  Nodes not used by a
    kept tet are dropped; nodes are numbered in lexicographic (x, y, z) order.
    Returns (nodes float64 (n,3), tets int32 (t,4)).
    """
    R = int(math.ceil(max(a, b, c))) + 2
    r = np.arange(-R, R + 1)
    I, J, K = (m.ravel() for m in np.meshgrid(r, r, r, indexing="ij"))
    lower = np.stack([I, J, K], 1).astype(np.float64)
    chunks = []
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = 1.0
        o = [d for d in range(3) if d != ax]
        c1 = lower + 0.5
        c2 = c1 + e
        face = lower.copy()
        face[:, ax] += 1.0
        corners = []
        for (u, v) in ((0, 0), (1, 0), (1, 1), (0, 1)):
            p = face.copy()
            p[:, o[0]] += u
            p[:, o[1]] += v
            corners.append(p)
        for q in range(4):
            pa, pb = corners[q], corners[(q + 1) % 4]
            cen = (c1 + c2 + pa + pb) / 4.0
            keep = (cen[:, 0] / a) ** 2 + (cen[:, 1] / b) ** 2 + (cen[:, 2] / c) ** 2 <= 1.0
            chunks.append(np.stack([c1[keep], c2[keep], pa[keep], pb[keep]], 1))
    T = np.concatenate(chunks)                       # (t, 4, 3) in half-units
    key = np.round(T.reshape(-1, 3) * 2).astype(np.int64)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    nodes = uniq.astype(np.float64) * (0.5 * h)
    tets = inv.reshape(-1, 4).astype(np.int32)
    # spatially coherent tet order: sort by centroid cell (x, y, z lexicographic)
    cen = nodes[tets].mean(1)
    cell = np.floor(cen / h).astype(np.int64)
    order = np.lexsort((cell[:, 2], cell[:, 1], cell[:, 0]))
    return nodes, tets[order]


def jitter(nodes: np.ndarray, frac: float, h: float, seed: int) -> np.ndarray:
    """Uniform jitter of +-frac*h per coordinate (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    return nodes + rng.uniform(-frac * h, frac * h, size=nodes.shape)


def single_tet() -> tuple[np.ndarray, np.ndarray]:
    """Unit right-corner tet."""
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64)
    return nodes, np.array([[0, 1, 2, 3]], np.int32)


def two_tet_fig4() -> tuple[np.ndarray, np.ndarray]:
    """Fig. 4 topology: A=(0,0,0) B=(1,0,0) C=(0,1,0) D=(0,0,1) E=(1,1,1);
    tets ABCD and BCDE share face BCD (node ids A..E = 0..4)."""
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    return nodes, tets


# --------------------------------------------------------------------------
# load cases
# --------------------------------------------------------------------------

def beam_config(jitter_seed: int = 0) -> Workload:
    """Three-point-bending beam: 4x4x16 unit cubes (1536 tets, 425 nodes).

    Supports: the bottom (y=0) node lines at z=1 and z=15 (x=0..4) pinned.
    Load: 500 N total along -y on the top (y=4) line at z=8, split over its
    5 nodes.  E=1e6 Pa, nu=0.3, rho=1000, dt=1e-3, 20 steps, threshold 0.5,
    non-local radius 1.5 edge lengths; +-1% node jitter with seed 0.
    """
    nodes, tets, grid = kuhn_box(4, 4, 16)
    nodes = jitter(nodes, 0.01, 1.0, jitter_seed)
    pinned = np.nonzero((grid[:, 1] == 0) & ((grid[:, 2] == 1) | (grid[:, 2] == 15)))[0].astype(np.int32)
    top = np.nonzero((grid[:, 1] == 4) & (grid[:, 2] == 8))[0]
    f = np.zeros_like(nodes)
    f[top, 1] = -500.0 / len(top)
    return Workload("beam_4x4x16_fp64", nodes, tets, 1e6, 0.3, 1000.0, 1e-3, 20, 0.5, 1.5, f, pinned)


LOAF_AXES = (39.5, 19.75, 15.8)


def _loaf_mesh(seed: int = 1):
    nodes, tets = bcc_ellipsoid(*LOAF_AXES)
    return jitter(nodes, 0.01, 1.0, seed), tets


def loaf_config(seed: int = 1, axes=LOAF_AXES) -> Workload:
    """Loaf stand-in: BCC lattice in an ellipsoid (39.5, 19.75, 15.8) cells.

    619,300 tets / 111,283 nodes / 746,378 edges at the default axes.  The
    two end caps (x within 10% of the length from either end) are pulled
    apart with 20 N per node along x.  Ductile E=2e4, nu=0.35, rho=1000,
    dt=5e-4, 200 steps, CG rel. tolerance 1e-6, R_d = 1.5 h.
    """
    nodes, tets = bcc_ellipsoid(*axes)
    nodes = jitter(nodes, 0.01, 1.0, seed)
    x = nodes[:, 0]
    L = x.max() - x.min()
    f = np.zeros_like(nodes)
    f[x <= x.min() + 0.1 * L, 0] = -20.0
    f[x >= x.max() - 0.1 * L, 0] = +20.0
    return Workload("loaf_bcc_620k_fp64", nodes, tets, 2e4, 0.35, 1000.0, 5e-4, 200,
                    LOAF_THRESHOLD, 1.5, f, np.zeros(0, np.int32))


# Driver threshold of the loaf case (dimensionless strain).  The configuration
# gives none; 1e-3 strain is the value used for it (the cost of a step does not
# depend on it).
LOAF_THRESHOLD = 1.0e-3


def glass_config(seed: int = 1, axes=LOAF_AXES) -> Workload:
    """Brittle glass on the loaf mesh: E=7e10, nu=0.22, rho=2500, dt=5e-4.

    A 1e4 N point impact (along -z) on the node nearest the top apex; the
    lowest 5% of nodes (by z) are pinned.  Mixed precision case.
    """
    nodes, tets = bcc_ellipsoid(*axes)
    nodes = jitter(nodes, 0.01, 1.0, seed)
    apex = int(np.argmax(nodes[:, 2] - 1e-3 * (np.abs(nodes[:, 0]) + np.abs(nodes[:, 1]))))
    f = np.zeros_like(nodes)
    f[apex, 2] = -1e4
    zcut = np.quantile(nodes[:, 2], 0.05)
    pinned = np.nonzero(nodes[:, 2] <= zcut)[0].astype(np.int32)
    return Workload("loaf_bcc_620k_glass_mixed", nodes, tets, 7e10, 0.22, 2500.0, 5e-4, 200,
                    GLASS_THRESHOLD, 1.5, f, pinned, precision="mixed")


GLASS_THRESHOLD = 1.0e-6


def batch_configs(n: int = 64, seed: int = 2, lo: float = 2e3, hi: float = 8e4) -> list[Workload]:
    """64 Kuhn boxes of uneven size: tet counts log-uniform in [2e3, 8e4].

    Each count is rounded to a box of 6*nx*ny*nz tets with nx = ny and
    nz = k*nx (aspect 1:1:k, k in {1..4} drawn with the same generator).
    Young's modulus log-uniform in [1e4, 1e8]; the bottom face (z=0) is
    pinned and a random force (seeded) acts on the top face nodes.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        k = int(rng.integers(1, 5))
        nx = max(1, int(round((target / (6.0 * k)) ** (1.0 / 3.0))))
        nodes, tets, grid = kuhn_box(nx, nx, k * nx)
        nodes = jitter(nodes, 0.01, 1.0, seed * 1000 + b)
        E = math.exp(rng.uniform(math.log(1e4), math.log(1e8)))
        f = np.zeros_like(nodes)
        top = np.nonzero(grid[:, 2] == k * nx)[0]
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        f[top] = direction * (E * 1e-4 * nx * nx / max(len(top), 1))
        pinned = np.nonzero(grid[:, 2] == 0)[0].astype(np.int32)
        out.append(Workload(f"box_{b}_{nx}x{nx}x{k*nx}", nodes, tets, E, 0.3, 1000.0, 1e-3, 20,
                            1e-2, 1.5, f, pinned, precision="mixed"))
    return out

"""CPU FP64 reference of the learned warm start and preconditioner (oracle).

Test infrastructure only (see the package docstring).  The paper has no
learned component; this module defines, in plain numpy, the message-passing
network the CUDA path trains and runs, so that its forward pass, loss and
gradients can be checked element by element.

Network (per node i, hidden width 64):
  h0   = relu(W0 f_i + b0)                                   node input f_i (16)
  for l = 1..3:
    a    = Wa_l h
    M_i  = (1/deg_i) sum_{j in N(i)} relu(a_j + We_l e_ij + bm_l)   edge input e_ij (16)
    h    = h + relu(Wu_l [h ; M] + bu_l)
  out_i = Wd h_i + bd                                         9 outputs: delta (3), ell (6)

Outputs (per node):
  L_i   = lower triangular, diagonal exp(ell_0..2), below (ell_3, ell_4, ell_5)
  P_i   = C_i (L_i L_i^T + eps I) C_i^T,  C_i C_i^T = D_i^-1 (Cholesky of the
          inverse diagonal block of A): symmetric positive definite, = block
          Jacobi scaled by (1 + eps) when L = I
  x0_i  = P_i b_i + s delta_i,  s = rms_i |D_i^-1 b_i|
Loss for a pair (b, x*) with A_ff x* = b on the free nodes f: the relative
error of x0 in the energy norm of the free block, which is the norm conjugate
gradients minimises,
  loss = (x0 - x*)^T A_ff (x0 - x*) / x*^T A_ff x*.
In a time step the network solves for the correction to the previous step's
solution x_prev: b = b_free - A_ff x_prev (``training_pair``) and the start
handed to the solver is x_prev + x0.

Weights are stored row-major as [in][out]; the forward pass uses them as given
(the GPU rounds them to bfloat16 first; tests pass the rounded values here).
"""
from __future__ import annotations

import numpy as np

HID = 64
NIN = 16
EIN = 16
NOUT = 9
EPS = 1e-3


def param_shapes():
    shapes = {"W0": (NIN, HID), "b0": (HID,)}
    for l in range(3):
        shapes.update({f"Wa{l}": (HID, HID), f"We{l}": (EIN, HID), f"bm{l}": (HID,),
                       f"Wu{l}": (2 * HID, HID), f"bu{l}": (HID,)})
    shapes.update({"Wd": (HID, NOUT), "bd": (NOUT,)})
    return shapes


def param_order():
    return list(param_shapes().keys())


def flatten(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k in param_order()])


def unflatten(vec) -> dict:
    out, o = {}, 0
    for k, shp in param_shapes().items():
        n = int(np.prod(shp))
        out[k] = np.asarray(vec[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def n_params() -> int:
    return sum(int(np.prod(s)) for s in param_shapes().values())


def block_inverse_cholesky(Ainv):
    """Lower Cholesky factor C of each 3x3 SPD block: C C^T = Ainv."""
    return np.linalg.cholesky(Ainv)


def lower_from_ell(ell):
    L = np.zeros(ell.shape[:-1] + (3, 3))
    L[..., 0, 0] = np.exp(ell[..., 0])
    L[..., 1, 1] = np.exp(ell[..., 1])
    L[..., 2, 2] = np.exp(ell[..., 2])
    L[..., 1, 0] = ell[..., 3]
    L[..., 2, 0] = ell[..., 4]
    L[..., 2, 1] = ell[..., 5]
    return L


class Graph:
    """Undirected mesh graph in CSR (no self loops) with per-directed-edge
    features e_ij for the message j -> i, stored at i's row."""

    def __init__(self, row_ptr, col, efeat):
        self.row_ptr = np.asarray(row_ptr, np.int64)
        self.col = np.asarray(col, np.int64)
        self.efeat = np.asarray(efeat, np.float64)        # (E, EIN)
        self.n = len(self.row_ptr) - 1
        self.dst = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        self.deg = np.maximum(np.diff(self.row_ptr), 1).astype(np.float64)


def forward(params, g: Graph, f, keep=False):
    """Returns the (n, 9) outputs (and the activations when keep=True)."""
    relu = lambda z: np.maximum(z, 0.0)
    z0 = f @ params["W0"] + params["b0"]
    h = relu(z0)
    cache = {"f": f, "z0": z0, "h": [h]}
    for l in range(3):
        a = h @ params[f"Wa{l}"]
        pre = a[g.col] + g.efeat @ params[f"We{l}"] + params[f"bm{l}"]     # (E, HID)
        msg = relu(pre)
        M = np.zeros_like(h)
        np.add.at(M, g.dst, msg)
        M /= g.deg[:, None]
        cat = np.concatenate([h, M], 1)
        zu = cat @ params[f"Wu{l}"] + params[f"bu{l}"]
        h = h + relu(zu)
        if keep:
            cache.setdefault("pre", []).append(pre)
            cache.setdefault("cat", []).append(cat)
            cache.setdefault("zu", []).append(zu)
        cache["h"].append(h)
    out = h @ params["Wd"] + params["bd"]
    return (out, cache) if keep else out


def apply_outputs(out, C, b, s):
    """P_i and x0_i from the network outputs (definitions in the module docstring)."""
    L = lower_from_ell(out[:, 3:9])
    G = L @ np.swapaxes(L, 1, 2) + EPS * np.eye(3)
    P = C @ G @ np.swapaxes(C, 1, 2)
    x0 = np.einsum("nab,nb->na", P, b) + s * out[:, 0:3]
    return P, x0, L, G


def loss_and_grad(params, g: Graph, f, C, b, dv, free, s, A):
    """Loss of one pair and d(loss)/d(params) by the chain rule (manual backward).
    A: the full system (scipy sparse, 3n x 3n); only its free block enters."""
    import scipy.sparse as sp
    out, cache = forward(params, g, f, keep=True)
    P, x0, L, G = apply_outputs(out, C, b, s)
    w = free.astype(np.float64)[:, None]
    A = sp.csr_matrix(A)
    e = (x0 - dv) * w
    q = (A @ e.ravel()).reshape(-1, 3) * w                     # A_ff e on free rows
    t = dv * w
    den = float(t.ravel() @ (A @ t.ravel()))
    if not den > 0:
        den = 1.0
    loss = float(e.ravel() @ q.ravel()) / den
    dx0 = 2.0 * q / den                                        # (n, 3)
    dout = np.zeros_like(out)
    dout[:, 0:3] = s * dx0
    dP = np.einsum("na,nb->nab", dx0, b)                       # d/dP of (P b)
    dG = np.swapaxes(C, 1, 2) @ dP @ C
    dL = (dG + np.swapaxes(dG, 1, 2)) @ L
    dout[:, 3] = dL[:, 0, 0] * L[:, 0, 0]
    dout[:, 4] = dL[:, 1, 1] * L[:, 1, 1]
    dout[:, 5] = dL[:, 2, 2] * L[:, 2, 2]
    dout[:, 6] = dL[:, 1, 0]
    dout[:, 7] = dL[:, 2, 0]
    dout[:, 8] = dL[:, 2, 1]
    grads = {k: np.zeros(v) for k, v in param_shapes().items()}
    h = cache["h"]
    grads["Wd"] = h[3].T @ dout
    grads["bd"] = dout.sum(0)
    dh = dout @ params["Wd"].T
    for l in reversed(range(3)):
        zu, cat, pre = cache["zu"][l], cache["cat"][l], cache["pre"][l]
        dzu = dh * (zu > 0)
        grads[f"Wu{l}"] = cat.T @ dzu
        grads[f"bu{l}"] = dzu.sum(0)
        dcat = dzu @ params[f"Wu{l}"].T
        dh_prev = dh + dcat[:, :HID]
        dM = dcat[:, HID:] / g.deg[:, None]
        dpre = dM[g.dst] * (pre > 0)                            # (E, HID)
        grads[f"We{l}"] = g.efeat.T @ dpre
        grads[f"bm{l}"] = dpre.sum(0)
        da = np.zeros_like(dh)
        np.add.at(da, g.col, dpre)
        grads[f"Wa{l}"] = h[l].T @ da
        dh = dh_prev + da @ params[f"Wa{l}"].T
    dz0 = dh * (cache["z0"] > 0)
    grads["W0"] = cache["f"].T @ dz0
    grads["b0"] = dz0.sum(0)
    return loss, grads


def init_params(seed: int) -> dict:
    """He-style random init; the decoder starts at zero (block-Jacobi start)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in param_shapes().items():
        if k.startswith("b") or k in ("Wd",):
            p[k] = np.zeros(shp)
        else:
            p[k] = rng.normal(size=shp) * np.sqrt(2.0 / shp[0])
    return p


def to_bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def build_inputs(A, mass, X, edges, pinned_mask, b):
    """Network inputs from an assembled system A (scipy sparse, 3n x 3n), the
    lumped mass, rest positions X, mesh edges (sorted (i, j) pairs), the
    pinned-node mask and the right-hand side b (n, 3).

    Node inputs f_i (16): [log(t_i / mean t), entries xx yy zz xy xz yz of
    A_ii / t_i - I, log(m_i / mean m), pinned flag, degree / 16,
    y_i / s (3), 0 0 0] with t_i = trace(A_ii) / 3, y_i = A_ii^-1 b_i on free
    nodes (0 on pinned ones) and s = sqrt(mean over free nodes of |y_i|^2).
    Edge inputs e_ij for the message j -> i (16): [(X_j - X_i) / mean rest edge
    length (3), A_ij / sqrt(t_i t_j) row-major (9), 0 0 0 0].
    Returns (Graph, f, C, s, free, Dinv)."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    n = X.shape[0]
    dd = np.zeros((n, 3, 3))
    idx = np.arange(n)
    for a in range(3):
        for c in range(3):
            dd[:, a, c] = np.asarray(A[3 * idx + a, 3 * idx + c]).ravel()
    t = np.trace(dd, axis1=1, axis2=2) / 3.0
    adj = [[] for _ in range(n)]
    for i, j in np.asarray(edges, np.int64):
        adj[i].append(j)
        adj[j].append(i)
    row_ptr = [0]
    col = []
    for i in range(n):
        col += sorted(adj[i])
        row_ptr.append(len(col))
    col = np.asarray(col, np.int64)
    dst = np.repeat(np.arange(n), np.diff(row_ptr))
    hbar = np.mean(np.linalg.norm(X[np.asarray(edges)[:, 1]] - X[np.asarray(edges)[:, 0]], axis=1))
    ef = np.zeros((len(col), EIN))
    ef[:, 0:3] = (X[col] - X[dst]) / hbar
    for a in range(3):
        for c in range(3):
            ef[:, 3 + 3 * a + c] = np.asarray(A[3 * dst + a, 3 * col + c]).ravel() / np.sqrt(t[dst] * t[col])
    free = ~np.asarray(pinned_mask, bool)
    Dinv = np.linalg.inv(dd)
    y = np.einsum("nab,nb->na", Dinv, b) * free[:, None]
    s = float(np.sqrt((y[free] ** 2).sum(1).mean())) if free.any() else 1.0
    if not s > 0:
        s = 1.0
    f = np.zeros((n, NIN))
    f[:, 0] = np.log(t / t.mean())
    rel = dd / t[:, None, None] - np.eye(3)
    for q, (a, c) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        f[:, 1 + q] = rel[:, a, c]
    f[:, 7] = np.log(mass / mass.mean())
    f[:, 8] = (~free).astype(np.float64)
    f[:, 9] = np.diff(row_ptr) / 16.0
    f[:, 10:13] = y / s
    g = Graph(row_ptr, col, ef)
    C = block_inverse_cholesky(Dinv)
    return g, f, C, s, free, Dinv


def training_pair(A, b, dv, x_prev, pinned_mask):
    """(b_net, target) of one solved step: with w = dv on pinned nodes and
    x_prev on free ones, b_net = b - A w on free rows (0 on pinned rows) and
    target = dv - x_prev on free nodes (0 on pinned).  b, dv, x_prev: (n, 3)."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    pin = np.asarray(pinned_mask, bool)
    wv = np.where(pin[:, None], dv, x_prev)
    bn = (b.ravel() - A @ wv.ravel()).reshape(-1, 3)
    bn[pin] = 0.0
    tg = np.where(pin[:, None], 0.0, dv - x_prev)
    return bn, tg

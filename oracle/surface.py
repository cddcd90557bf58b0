"""Split visualisation mesh of Sec. 4.1 (oracle; output only).

The computational mesh is never remeshed.  For display, every tet is cut into
the four node-associated pieces of Fig. 6c: the piece of node a holds a, the
midpoints of a's three edges, the centroids of a's three faces and the tet
centroid.  An edge splits into two child nodes at its midpoint, a face into
three at its centroid, a tet into four at its centroid, one child per parent
node of the entity.  Children take no part in the dynamics.  A child follows
the parents it is still joined to through unbroken edges of its own entity.
Sec. 4.1 works this through for a face: with edges (1,2) and (1,3) broken and
(2,3) whole, child 1 follows parent 1, and children 2 and 3 follow the
average movement of parents 2 and 3.

Reading taken: to "follow" is to sit at the entity's rest centroid plus the
mean displacement x - X of the joined parents.  An entity with no broken edge
therefore has all its children at its current centroid, with no gap.

Vertex numbering of the output (float64 [n_vertices][3]):
  [0, N)                     the nodes' current positions x;
  N + 2 e + s                child of edge e at its node edges[e][s];
  N + 2 NE + 3 f + c         child of face f at its c-th node (faces[f] sorted);
  N + 2 NE + 3 NF + 4 t + a  child of tet t at its local node a.
Crack surface: for every tet t and every broken local edge k = (a, b) (Eq. 21
labels), with c < d the tet's other two local nodes, two quads on the
interface of the pieces of a and b:
  [E(k, a), F(abc, a), T(t, a), F(abd, a)]  and  [E(k, b), F(abd, b), T(t, b), F(abc, b)],
listed by tet, then local edge, a-side first.
"""
from __future__ import annotations

import numpy as np

from .mesh import LOCAL_EDGES

# local faces: face i is opposite local node i
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def faces_of(tets: np.ndarray):
    """Unique faces as sorted node triples (lexicographic) and tet_faces (t, 4):
    the face opposite each local node."""
    tets = np.asarray(tets, np.int64)
    tri = np.stack([tets[:, list(f)] for f in LOCAL_FACES], 1)        # (t, 4, 3)
    tri = np.sort(tri, axis=2)
    faces, inv = np.unique(tri.reshape(-1, 3), axis=0, return_inverse=True)
    return faces, inv.reshape(-1, 4)


def _components(nodes, broken):
    """Labels of the connected components of `nodes` joined by the unbroken
    edges among them; broken(u, v) says whether edge (u, v) is broken."""
    comp = list(range(len(nodes)))

    def find(i):
        while comp[i] != i:
            i = comp[i]
        return i

    for i in range(len(nodes)):
        for j in range(i + 1, len(nodes)):
            if not broken(nodes[i], nodes[j]):
                ri, rj = find(i), find(j)
                if ri != rj:
                    comp[max(ri, rj)] = min(ri, rj)
    return [find(i) for i in range(len(nodes))]


def _follow(X, x, nodes, broken):
    """Child positions of one entity: rest centroid + mean displacement of the
    joined parents, one child per node (in the order of `nodes`)."""
    Xc = X[list(nodes)].mean(0)
    comp = _components(nodes, broken)
    out = np.zeros((len(nodes), 3))
    for i in range(len(nodes)):
        grp = [nodes[j] for j in range(len(nodes)) if comp[j] == comp[i]]
        out[i] = Xc + (x[grp] - X[grp]).mean(0)
    return out


def surface(X, x, tets, edges, labels):
    """(vertices float64 [N + 2 NE + 3 NF + 4 T][3], quads int64 [Q][4], faces, tet_faces)."""
    X, x = np.asarray(X, np.float64), np.asarray(x, np.float64)
    tets = np.asarray(tets, np.int64)
    edges = np.asarray(edges, np.int64)
    N, NE, T = len(X), len(edges), len(tets)
    eid = {(int(a), int(b)): k for k, (a, b) in enumerate(edges)}
    lab = np.asarray(labels).astype(bool)

    def broken(u, v):
        return bool(lab[eid[(min(u, v), max(u, v))]])

    faces, tet_faces = faces_of(tets)
    NF = len(faces)
    verts = np.zeros((N + 2 * NE + 3 * NF + 4 * T, 3))
    verts[:N] = x
    for e, (a, b) in enumerate(edges):
        verts[N + 2 * e:N + 2 * e + 2] = _follow(X, x, (int(a), int(b)), broken)
    o = N + 2 * NE
    for f, tri in enumerate(faces):
        verts[o + 3 * f:o + 3 * f + 3] = _follow(X, x, tuple(int(v) for v in tri), broken)
    o2 = o + 3 * NF
    for t in range(T):
        verts[o2 + 4 * t:o2 + 4 * t + 4] = _follow(X, x, tuple(int(v) for v in tets[t]), broken)
    quads = []
    for t in range(T):
        for k, (a, b) in enumerate(LOCAL_EDGES):
            na, nb = int(tets[t, a]), int(tets[t, b])
            e = eid[(min(na, nb), max(na, nb))]
            if not lab[e]:
                continue
            c, d = [v for v in range(4) if v not in (a, b)]
            f_abc, f_abd = tet_faces[t, d], tet_faces[t, c]

            def E(node):
                return N + 2 * e + (0 if edges[e, 0] == node else 1)

            def F(f, node):
                return o + 3 * f + int(np.nonzero(faces[f] == node)[0][0])

            quads.append([E(na), F(f_abc, na), o2 + 4 * t + a, F(f_abd, na)])
            quads.append([E(nb), F(f_abd, nb), o2 + 4 * t + b, F(f_abc, nb)])
    return verts, np.array(quads, np.int64).reshape(-1, 4), faces, tet_faces

"""Hand derivation of ``nonlocal_chi_lag.json`` in exact rational arithmetic.

Four disjoint right-corner tets (corner o, legs a along x, y, z; node order
corner, +x, +y, +z) with rest centroids o + a/4 (1, 1, 1).  Every quantity
below is a closed form of the paper's definitions, evaluated with fractions;
nothing here imports the oracle or the CUDA library.

* Eq. 20 weight (reading: V_j (1 - r^2/R_d^2)^2 over REST centroids,
  normalised to sum 1).  With R_d = 2 the squared centroid distances are
  0, 1, 2, 3, 2.25 (and 6.25, 8.25 outside the ball), so every weight is a
  small fraction.
* Homogeneous stretch F = diag(f) of a tet gives the Green strain
  e = (f^2 - 1)/2 along the stretched axis, and StVK (Eq. 37) gives
  S = lam e I + 2 mu e (axis) with E = 1, nu = 1/4: lam = mu = 2/5.
* The normal stress of Eq. 16-19 along a current unit edge n of a diagonal
  S is sum_i S_ii n_i^2 (no shear terms, so the shear coefficient drops out).
  A corner tet stretched by diag(fx, fy, fz) has current edge directions
  (fx,0,0) (0,fy,0) (0,0,fz) (-fx,fy,0) (-fx,0,fz) (0,-fy,fz) for its six
  local edges in the order of Eq. 15.
* Eq. 21: an edge breaks when its driver sigma*/E reaches theta = 1/4, and
  stays broken.  Eq. 25: chi = sum over unbroken edges of |sigma_f| over the
  sum over all six, with the tet's own sigma_f = T S (chi = 1 with no broken
  edge).
* Step 2 averages chi_j S_j with the chi of step 1 (the previous step).

Run it to print the JSON that is stored beside it.
"""
from fractions import Fraction as Fr
import json

LAM = MU = Fr(2, 5)
R_D = Fr(2)
THETA = Fr(1, 4)
CORNERS = [(Fr(0), Fr(0), Fr(0)), (Fr(9, 10), Fr(-1, 10), Fr(-1, 10)), (Fr(0), Fr(1), Fr(1)), (Fr(5, 2), Fr(0), Fr(0))]
LEGS = [Fr(2, 5), Fr(4, 5), Fr(2, 5), Fr(2, 5)]
# step 1: tet k stretched along x by STRETCH1[k] about its corner; step 2: tet 1
# stretched along y by 13/10 instead; tet 2 is also translated rigidly by
# (0, 3, 0) in both steps (it moves the CURRENT centroids only)
STRETCH1 = [(Fr(11, 10), 1, 1), (Fr(12, 10), 1, 1), (Fr(9, 10), 1, 1), (Fr(13, 10), 1, 1)]
STRETCH2 = [STRETCH1[0], (1, Fr(13, 10), 1), STRETCH1[2], STRETCH1[3]]
TRANSLATE = [(0, 0, 0), (0, 0, 0), (0, 3, 0), (0, 0, 0)]


def weights():
    vol = [a ** 3 / 6 for a in LEGS]
    cen = [tuple(o[i] + a / 4 for i in range(3)) for o, a in zip(CORNERS, LEGS)]
    out = []
    for ce in cen:
        raw = {}
        for j, cj in enumerate(cen):
            r2 = sum((p - q) ** 2 for p, q in zip(ce, cj))
            if r2 <= R_D ** 2:
                raw[j] = vol[j] * (1 - r2 / R_D ** 2) ** 2
        tot = sum(raw.values())
        out.append({j: w / tot for j, w in raw.items()})
    return out


def stress(f):
    """Diagonal of S for the stretch diag(f) (one stretched axis)."""
    d = []
    for i in range(3):
        e = (Fr(f[i]) ** 2 - 1) / 2
        d.append(e)
    tr = sum(d)
    return [LAM * tr + 2 * MU * d[i] for i in range(3)]


def edge_normal(Sd, f):
    fx, fy, fz = (Fr(c) for c in f)
    dirs = [(fx, 0, 0), (0, fy, 0), (0, 0, fz), (-fx, fy, 0), (-fx, 0, fz), (0, -fy, fz)]
    return [sum(Sd[i] * d[i] ** 2 for i in range(3)) / sum(c ** 2 for c in d) for d in dirs]


def damage_step(W, stretch, chi_prev, broken_prev):
    S = [stress(f) for f in stretch]
    sbar = [[sum(w * chi_prev[j] * S[j][i] for j, w in W[e].items()) for i in range(3)] for e in range(4)]
    drv = [edge_normal(sbar[e], stretch[e]) for e in range(4)]          # E = 1: driver = sigma*
    broken = [[broken_prev[e][k] or drv[e][k] >= THETA for k in range(6)] for e in range(4)]
    chi = []
    for e in range(4):
        sf = edge_normal(S[e], stretch[e])
        if not any(broken[e]):
            chi.append(Fr(1))
        else:
            chi.append(sum(abs(v) for v, b in zip(sf, broken[e]) if not b) / sum(abs(v) for v in sf))
    return sbar, drv, broken, chi


def main():
    W = weights()
    s1 = damage_step(W, STRETCH1, [Fr(1)] * 4, [[False] * 6 for _ in range(4)])
    s2 = damage_step(W, STRETCH2, s1[3], s1[2])
    flt = lambda rows: [[float(v) for v in r] for r in rows]
    out = {"_source": "Hand-worked Eq. 20 weights and the chi lag of the Eq. 20 average (readings: weight "
                      "V_j (1 - r^2/R_d^2)^2 over rest centroids, normalised; step 2 averages chi_j S_j with step "
                      "1's chi). Four disjoint right-corner tets, E = 1, nu = 1/4 (lam = mu = 2/5), R_d = 2, "
                      "theta = 1/4 (strain driver), shear coefficient irrelevant (diagonal stresses). Exact "
                      "fractions in tests/golden/derive_nonlocal_chi_lag.py; Sec. 3.3, Eq. 14-25.",
           "corners": [[float(c) for c in o] for o in CORNERS], "legs": [float(a) for a in LEGS],
           "stretch_step1": [[float(c) for c in f] for f in STRETCH1],
           "stretch_step2": [[float(c) for c in f] for f in STRETCH2],
           "translate": [[float(c) for c in t] for t in TRANSLATE],
           "young": 1.0, "poisson": 0.25, "radius": float(R_D), "threshold": float(THETA),
           "weights": [{str(j): str(w) for j, w in we.items()} for we in W]}
    for k, (sbar, drv, broken, chi) in enumerate((s1, s2), 1):
        out[f"step{k}"] = {"sigma_bar_diag": flt(sbar), "driver": [float(v) for r in drv for v in r],
                           "broken": [int(b) for r in broken for b in r], "chi": [float(c) for c in chi]}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()

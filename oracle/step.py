"""One implicit time step of graph-based FEM fracture (oracle).

Order of Algorithm 1 (Sec. 4.3), minus the visualisation remesh and the
collision response, which are not part of the computational step:
  1. stresses along the edges at the start-of-step positions, non-local
     average, fracture check and relabel (Eq. 14-21), then chi (Eq. 22-25);
  2. build the system with f* = chi f and K* = sum chi k (Eq. 32-34), mass
     (Eq. 5, row-sum lumped by default) and damping b* = alpha m + beta k*
     (Sec. 3.6);
  3. solve for the velocity (implicit backward Euler + CG, Sec. 4.3);
  4. x += dt v.

The backward-Euler update is linearised once about the start of the step
(one Newton iteration), with unknown dv = v_{n+1} - v_n:
  [(1 + dt alpha) M + (dt beta + dt^2) K*] dv
      = dt [ f_ext + f*(x_n) - alpha M v_n - (beta + dt) K* v_n ]
which is Eq. 2 with f_int(x_{n+1}) ~ f_int(x_n) + K* dt v_{n+1}.
Pinned nodes have all three velocity components prescribed (zero by default).

More Newton iterations (``newton_iters`` > 1) solve the backward-Euler
residual itself,
  r(v) = M (v - v_n) + dt (B v - f_ext - f*(x_n + dt v)),
  B = alpha M + beta K*(x),
from the guess v^0 = 0 (so that x^0 = x_n and the first iterate is the
linearised step above): J_k = M + dt B_k + dt^2 K*(x^k), J_k d = -r(v^k),
v^{k+1} = v^k + d, with the damping matrix taken at the current iterate and
chi frozen for the step.  ``mass="consistent"`` uses the element masses of
Eq. 5 as they stand instead of their row sums.

``quasistatic_step`` is the paper's quasi-static solve (Eq. 36, Sec. 4.3): no
mass or damping, the equilibrium f*(x) + f_ext = 0 on free DOFs found by
Newton's method with a backtracking line search on the total energy
E(x) = sum_e chi_e V_e Psi_e(x) - f_ext . x.  The damage update comes first, at
the start-of-step positions (the order of Algorithm 1), then the pinned nodes
move to their prescribed positions and chi stays frozen for the solve.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import damage, elastic, mesh, solve


@dataclasses.dataclass
class Material:
    young: float
    poisson: float
    density: float
    threshold: float = np.inf
    radius: float = 0.0
    alpha: float = 0.0
    beta: float = 0.0
    driver_mode: str = "strain"       # "strain" (sigma*/E) or "stress"
    shear_coef: float = 2.0           # 2: tensor n.S.n; 1: Eq. 16 as printed
    average_degraded: bool = True     # Eq. 20 averages chi_j S_j (True) or S_j
    mass: str = "lumped"              # "lumped" (row sums of Eq. 5) or "consistent" (Eq. 5)
    energy: str = "stvk"              # "stvk" (Eq. 37) or "snh" (Eq. 35, squared reading)


@dataclasses.dataclass
class State:
    x: np.ndarray          # (n, 3)
    v: np.ndarray          # (n, 3)
    labels: np.ndarray     # (ne,) uint8, 1 = broken
    chi: np.ndarray        # (t,) energy degradation in force during the last step


class Model:
    """Rest-state precompute of one mesh (Sec. 3.1-3.3)."""

    def __init__(self, nodes, tets, mat: Material, nonlocal_lists=True):
        self.X = np.asarray(nodes, np.float64)
        self.tets = np.asarray(tets, np.int64)
        self.mat = mat
        self.lam, self.mu = elastic.lame(mat.young, mat.poisson)
        self.edges, self.tet_edges = mesh.edges_of(self.tets)
        self.V, self.D2, self.q = mesh.rest_geometry(self.X, self.tets)
        self.mass = mesh.lumped_mass(self.X, self.tets, mat.density, self.V)
        if mat.mass == "consistent":
            self.M = mesh.consistent_mass_matrix(self.X, self.tets, mat.density, self.V)
        elif mat.mass == "lumped":
            self.M = sp.diags(np.repeat(self.mass, 3)).tocsr()
        else:
            raise ValueError(f"unknown mass matrix {mat.mass!r}")
        self.centroids = mesh.centroids(self.X, self.tets)
        self.nbrs = self.weights = None
        if nonlocal_lists:
            self.nbrs = mesh.nonlocal_neighbours(self.X, self.tets, mat.radius)
            self.weights = damage.nonlocal_weights(self.centroids, self.V, self.nbrs, mat.radius)

    @property
    def n_nodes(self):
        return self.X.shape[0]

    def rest_state(self) -> State:
        return State(self.X.copy(), np.zeros_like(self.X), np.zeros(len(self.edges), np.uint8),
                     np.ones(len(self.tets)))

    # ---- damage (Eq. 14-25) ------------------------------------------------
    def stresses(self, x):
        """Per-tet S (Voigt, Eq. 14) and local edge-normal stress sigma_f = T S (Eq. 18)."""
        s = elastic.squared_edge_lengths(x, self.tets)
        C = elastic.cauchy_green_lsq(s, self.D2, self.q)
        J = None
        if self.mat.energy == "snh":
            J = elastic.orientation(x, self.tets, self.q) * np.sqrt(np.linalg.det(C))
        S = damage.stress_voigt(C, self.lam, self.mu, self.mat.energy, J)
        T = damage.projection_T(x, self.tets, self.mat.shear_coef)
        return S, T, np.einsum("tkc,tc->tk", T, S)

    def damage_update(self, state: State):
        """Returns (driver per edge, new labels, new chi, sigma* per (tet, edge))."""
        S, T, sigf = self.stresses(state.x)
        sig_in = S * state.chi[:, None] if self.mat.average_degraded else S
        sig_bar = damage.nonlocal_average(sig_in, self.nbrs, self.weights)     # Eq. 20 sum
        sig_star = np.einsum("tkc,tc->tk", T, sig_bar)                          # Eq. 20 T(...)
        drv = damage.edge_driver(sig_star, self.tet_edges, len(self.edges), self.mat.young,
                                 self.mat.driver_mode)
        labels = damage.relabel(state.labels, drv, self.mat.threshold)          # Eq. 21
        chi = damage.chi(labels, self.tet_edges, sigf, self.mat.young)          # Eq. 25
        return drv, labels, chi, sig_star

    def chi_from_labels(self, x, labels):
        """chi of Eq. 25 for given labels at positions x."""
        _, _, sigf = self.stresses(x)
        return damage.chi(labels, self.tet_edges, sigf, self.mat.young)

    # ---- system (Eq. 2, 32-34) ---------------------------------------------
    def assemble(self, x, chi):
        """Global K* = sum chi k_e (Eq. 34, CSR) and f* = sum chi f_e (Eq. 32)."""
        Ke = elastic.element_tangent(x, self.tets, self.V, self.D2, self.q, self.lam, self.mu, chi, self.mat.energy)
        fe = elastic.element_forces(x, self.tets, self.V, self.D2, self.q, self.lam, self.mu, chi, self.mat.energy)
        dof = (3 * self.tets[:, :, None] + np.arange(3)).reshape(-1, 12)
        rows = np.repeat(dof, 12, axis=1).ravel()
        cols = np.tile(dof, (1, 12)).ravel()
        n3 = 3 * self.n_nodes
        K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n3, n3)).tocsr()
        f = np.zeros(n3)
        np.add.at(f, dof.ravel(), fe.reshape(-1))
        return K, f

    def linear_system(self, x, v, chi, dt, f_ext):
        """A dv = b of the linearised backward-Euler step (module docstring)."""
        mt = self.mat
        K, f = self.assemble(x, chi)
        M = self.M
        A = ((1.0 + dt * mt.alpha) * M + (dt * mt.beta + dt * dt) * K).tocsr()
        vv = v.ravel()
        b = dt * (np.asarray(f_ext, np.float64).ravel() + f - mt.alpha * (M @ vv)
                  - (mt.beta + dt) * (K @ vv))
        return A, b, K, f

    def newton_residual(self, x_n, v_n, v, chi, dt, f_ext):
        """r(v) of the backward-Euler step (module docstring) with B at x = x_n + dt v,
        and its Jacobian J = M + dt B + dt^2 K*(x)."""
        mt = self.mat
        x = x_n + dt * v.reshape(-1, 3)
        K, f = self.assemble(x, chi)
        B = mt.alpha * self.M + mt.beta * K
        vv, vn = v.ravel(), v_n.ravel()
        r = self.M @ (vv - vn) + dt * (B @ vv - np.asarray(f_ext, np.float64).ravel() - f)
        J = (self.M + dt * B + dt * dt * K).tocsr()
        return r, J

    def step(self, state: State, dt: float, f_ext, pinned=None, pinned_vel=None,
             solver: str = "direct", rtol: float = 1e-13, maxit: int = 100000, newton_iters: int = 1):
        """One step; returns (new State, info dict)."""
        if newton_iters > 1:
            return self.step_newton(state, dt, f_ext, pinned, pinned_vel, newton_iters, solver, rtol, maxit)
        drv, labels, chi, sig_star = self.damage_update(state)
        A, b, K, f = self.linear_system(state.x, state.v, chi, dt, f_ext)
        n = self.n_nodes
        fixed = np.zeros(n, bool)
        dv = np.zeros(3 * n)
        if pinned is not None and len(pinned):
            pinned = np.asarray(pinned, np.int64)
            fixed[pinned] = True
            target = np.zeros((len(pinned), 3)) if pinned_vel is None else np.asarray(pinned_vel).reshape(-1, 3)
            dv.reshape(-1, 3)[pinned] = target - state.v[pinned]
        free = np.repeat(~fixed, 3)
        rhs = b[free] - A[free][:, ~free] @ dv[~free]
        Aff = A[free][:, free].tocsr()
        info = {"driver": drv, "labels": labels, "chi": chi, "sig_star": sig_star, "A": A, "b": b,
                "K": K, "f": f}
        if solver == "direct":
            dv[free] = solve.direct(Aff, rhs) if rhs.size else rhs
            info.update(iters=0, status="ok")
        else:
            sol, it, rel, status = solve.pcg(Aff, rhs, rtol=rtol, maxit=maxit)
            dv[free] = sol
            info.update(iters=it, rel_res=rel, status=status)
        rn = np.linalg.norm(rhs)
        info["rel_res"] = np.linalg.norm(rhs - Aff @ dv[free]) / rn if rn > 0 else 0.0
        v_new = state.v + dv.reshape(-1, 3)
        x_new = state.x + dt * v_new
        info["dv"] = dv.reshape(-1, 3)
        return State(x_new, v_new, labels, chi), info

    def step_newton(self, state: State, dt: float, f_ext, pinned, pinned_vel, iters: int,
                    solver: str = "direct", rtol: float = 1e-13, maxit: int = 100000):
        """Backward Euler by Newton's method on r(v) (module docstring): the damage
        update once at x_n, then `iters` Newton iterations from v^0 = 0 with
        the pinned velocities imposed from the first iteration on."""
        drv, labels, chi, sig_star = self.damage_update(state)
        n = self.n_nodes
        fixed = np.zeros(n, bool)
        vp = np.zeros((0, 3))
        if pinned is not None and len(pinned):
            pinned = np.asarray(pinned, np.int64)
            fixed[pinned] = True
            vp = np.zeros((len(pinned), 3)) if pinned_vel is None else np.asarray(pinned_vel).reshape(-1, 3)
        free = np.repeat(~fixed, 3)
        v = np.zeros(3 * n)
        res, iters_cg = [], 0
        for k in range(iters):
            r, J = self.newton_residual(state.x, state.v, v, chi, dt, f_ext)
            d = np.zeros(3 * n)
            if fixed.any():
                d.reshape(-1, 3)[fixed] = vp - v.reshape(-1, 3)[fixed]
            rhs = -r[free] - J[free][:, ~free] @ d[~free]
            res.append(float(np.linalg.norm(rhs)))
            Jff = J[free][:, free].tocsr()
            if solver == "direct":
                d[free] = solve.direct(Jff, rhs) if rhs.size else rhs
            else:
                sol, it, _, _ = solve.pcg(Jff, rhs, rtol=rtol, maxit=maxit)
                d[free] = sol
                iters_cg += it
            v = v + d
        r, _ = self.newton_residual(state.x, state.v, v, chi, dt, f_ext)
        v_new = v.reshape(-1, 3)
        x_new = state.x + dt * v_new
        info = {"driver": drv, "labels": labels, "chi": chi, "sig_star": sig_star, "dv": v_new - state.v,
                "newton_res": res, "final_res": float(np.linalg.norm(r[free])), "iters": iters_cg}
        return State(x_new, v_new, labels, chi), info

    def total_energy(self, x, chi, f_ext, with_scale=False):
        """E(x) = sum_e chi_e V_e Psi_e(x) - f_ext . x (the quasi-static objective);
        with_scale also returns sum |chi V Psi| + sum |f_i x_i|, the magnitude that
        sets the rounding of E."""
        psi = elastic.element_energy(x, self.tets, self.V, self.D2, self.q, self.lam, self.mu, chi, self.mat.energy)
        fx = np.asarray(f_ext, np.float64).ravel() * x.ravel()
        e = float(psi.sum() - fx.sum())
        return (e, float(np.abs(psi).sum() + np.abs(fx).sum())) if with_scale else e

    def quasistatic_step(self, state: State, f_ext, pinned=None, pinned_pos=None, max_newton: int = 50,
                         rtol: float = 1e-10, c_armijo: float = 1e-4):
        """Quasi-static load step (module docstring).  Newton direction K*_ff d = r_f
        with r = f_ext + f*(x); step length by halving from 1 until
        E(x + a d) <= E(x) - c a r.d.  Stops when |r_f| <= rtol |r_f at the start|.
        Returns (new State with v = 0, info)."""
        drv, labels, chi, sig_star = self.damage_update(state)
        n = self.n_nodes
        x = state.x.copy()
        fixed = np.zeros(n, bool)
        if pinned is not None and len(pinned):
            pinned = np.asarray(pinned, np.int64)
            fixed[pinned] = True
            if pinned_pos is not None:
                x[pinned] = np.asarray(pinned_pos, np.float64).reshape(-1, 3)
        free = np.repeat(~fixed, 3)
        fe = np.asarray(f_ext, np.float64).ravel()
        res, alphas, energies = [], [], []
        r0 = None
        for k in range(max_newton):
            K, f = self.assemble(x, chi)
            r = (fe + f)[free]
            rn = float(np.linalg.norm(r))
            res.append(rn)
            if r0 is None:
                r0 = rn
            if rn <= rtol * r0 or rn == 0.0:
                break
            d = np.zeros(3 * n)
            d[free] = solve.direct(K[free][:, free].tocsr(), r)
            slope = float(r @ d[free])
            e0, scale = self.total_energy(x, chi, fe, with_scale=True)
            energies.append(e0)
            a = 1.0
            while a > 2.0 ** -30:
                if c_armijo * a * slope <= 1e-12 * scale:
                    break
                if self.total_energy(x + a * d.reshape(-1, 3), chi, fe) <= e0 - c_armijo * a * slope:
                    break
                a *= 0.5
            alphas.append(a)
            x = x + a * d.reshape(-1, 3)
        info = {"driver": drv, "labels": labels, "chi": chi, "sig_star": sig_star, "newton_res": res,
                "alphas": alphas, "energies": energies}
        return State(x, np.zeros_like(state.v), labels, chi), info

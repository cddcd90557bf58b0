"""Thin Python binding of the graph-FEM fracture C ABI (include/graphfem.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Host arrays (numpy, or CPU torch tensors) are passed as GF_MEM_HOST; CUDA
torch tensors as GF_MEM_DEVICE.  By default the library allocates through
torch's caching allocator and runs on torch's current stream, so torch is the
device-memory and stream plumbing.  There is no CPU fallback: without the
built library or a CUDA device, calls raise.
"""
from __future__ import annotations

import atexit
import ctypes
import json
import weakref
import math
import os
import time
from typing import Optional

import numpy as np

from . import build as _build

MEM_HOST, MEM_DEVICE = 0, 1
DRIVER_STRAIN, DRIVER_STRESS = 0, 1
FP64, MIXED = 0, 1

STATUS = {0: "ok", 1: "bad argument", 2: "CUDA error", 3: "CG breakdown", 4: "CG max iterations", 5: "non-finite",
          6: "timeout", 7: "out of memory", 8: "unsupported"}


# Live handles, closed at interpreter exit (batches before the meshes they step,
# learned models before theirs) while the allocator callbacks into torch still
# work; a destroy left to __del__ during finalisation can call a freed callback.
_LIVE = {"batch": weakref.WeakSet(), "gnn": weakref.WeakSet(), "mesh": weakref.WeakSet()}


@atexit.register
def _close_live():
    for kind in ("batch", "gnn", "mesh"):
        for obj in list(_LIVE[kind]):
            try:
                obj.close()
            except Exception:
                pass


class GraphFEMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(ctypes.Structure):
    _fields_ = [("young", ctypes.c_double), ("poisson", ctypes.c_double), ("density", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("threshold", ctypes.c_double),
                ("radius", ctypes.c_double), ("driver_mode", ctypes.c_int32), ("shear_coef", ctypes.c_int32),
                ("average_degraded", ctypes.c_int32), ("mass_matrix", ctypes.c_int32), ("energy", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("cg_maxit", ctypes.c_int32), ("cg_rtol", ctypes.c_double),
                ("precond", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cg_iters", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("n_broken", ctypes.c_int64), ("n_new_broken", ctypes.c_int64), ("n_chi_zero", ctypes.c_int64),
                ("refine_sweeps", ctypes.c_int32), ("newton_iters", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("assembly", ctypes.c_int32), ("step_launch", ctypes.c_int32), ("solve_loop", ctypes.c_int32),
                ("wait_test", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


ASSEMBLY_GATHER, ASSEMBLY_COLOUR = 0, 1
STEP_GRAPH, STEP_STREAM = 0, 1
SOLVE_KERNELS, SOLVE_PERSISTENT, SOLVE_CG, SOLVE_DISTRIBUTED, SOLVE_NESTED = 0, 1, 2, 3, 4
QS_SOLVE_FP64, QS_SOLVE_NESTED = 0, 1


class BatchTuning(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("chunk", ctypes.c_int32), ("grid_budget", ctypes.c_int32),
                ("solve_loop", ctypes.c_int32), ("inner", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class MeshInfo(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("n_nodes", "n_tets", "n_edges", "n_blocks", "n_colours",
                                              "n_nbr_pairs", "device_bytes", "n_joint_entries", "n_union_rows",
                                              "eq20_tile")]


_LIB = None
P = ctypes.c_void_p


def metrics_line(step: int, dt: float, status: int, stats: dict) -> str:
    """One JSON line of the per-step metrics log."""
    rec = {"step": int(step), "time": time.time(), "dt": float(dt), "status": int(status)}
    rec.update({k: (float(v) if isinstance(v, float) else int(v)) for k, v in stats.items()})
    return json.dumps(rec, sort_keys=True)


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the built shared library (building it first if the sources are newer)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    sig = {
        "gf_mesh_create": (ctypes.c_int, [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.POINTER(Material),
                                          ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "gf_mesh_destroy": (None, [P]),
        "gf_mesh_plan": (ctypes.c_int, [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.POINTER(Material),
                                        ctypes.POINTER(MeshInfo), P, P, P]),
        "gf_mesh_info_get": (ctypes.c_int, [P, ctypes.POINTER(MeshInfo)]),
        "gf_state_set": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int32]),
        "gf_step": (ctypes.c_int, [P, ctypes.c_double, P, P, ctypes.c_int64, P, ctypes.c_int32,
                                   ctypes.POINTER(StepStats)]),
        "gf_solver_set": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_int32]),
        "gf_threshold_set": (ctypes.c_int, [P, ctypes.c_double]),
        "gf_refine_set": (ctypes.c_int, [P, ctypes.c_double]),
        "gf_quasistatic_solver_set": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_double]),
        "gf_mesh_autotune": (ctypes.c_int, [P, ctypes.c_double, P, P, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int32,
                                            P, P]),
        "gf_newton_set": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_double]),
        "gf_surface_sizes": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]),
        "gf_surface_get": (ctypes.c_int, [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
        "gf_quasistatic_step": (ctypes.c_int, [P, P, P, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_double, ctypes.POINTER(StepStats)]),
        "gf_tuning_set": (ctypes.c_int, [P, ctypes.POINTER(Tuning)]),
        "gf_tuning_get": (ctypes.c_int, [P, ctypes.POINTER(Tuning)]),
        "gf_positions_get": (ctypes.c_int, [P, P, ctypes.c_int32]),
        "gf_velocities_get": (ctypes.c_int, [P, P, ctypes.c_int32]),
        "gf_damage_get": (ctypes.c_int, [P, P, P, ctypes.c_int32]),
        "gf_chi_get": (ctypes.c_int, [P, P, ctypes.c_int32]),
        "gf_edges_get": (ctypes.c_int, [P, P]),
        "gf_system_get": (ctypes.c_int, [P, P, P, P, P]),
        "gf_profile_enable": (ctypes.c_int, [P, ctypes.c_int32]),
        "gf_profile_get": (ctypes.c_int32, [P, P, P, ctypes.c_int32]),
        "gf_profile_name": (ctypes.c_char_p, [ctypes.c_int32]),
        "gf_profile_reset": (ctypes.c_int, [P]),
        "gf_launch_count": (ctypes.c_int64, [P]),
        "gf_bsr_pcg_solve_static": (ctypes.c_int, [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_double,
                                                   ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int32),
                                                   ctypes.POINTER(ctypes.c_double)]),
        "gf_batch_create": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(P)]),
        "gf_batch_destroy": (None, [P]),
        "gf_batch_step": (ctypes.c_int, [P, ctypes.c_double, P, P, P, P, ctypes.c_int32, P]),
        "gf_batch_tuning_set": (ctypes.c_int, [P, ctypes.POINTER(BatchTuning)]),
        "gf_batch_tuning_get": (ctypes.c_int, [P, ctypes.POINTER(BatchTuning)]),
        "gf_batch_autotune": (ctypes.c_int, [P, ctypes.c_double, P, P, P, P, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(BatchTuning), ctypes.POINTER(ctypes.c_double)]),
        "gf_batch_launch_count": (ctypes.c_int64, [P]),
        "gf_gnn_n_params": (ctypes.c_int64, []),
        "gf_gnn_create": (ctypes.c_int, [P, ctypes.POINTER(P)]),
        "gf_gnn_destroy": (None, [P]),
        "gf_gnn_params_set": (ctypes.c_int, [P, P, ctypes.c_int64]),
        "gf_gnn_params_get": (ctypes.c_int, [P, P, ctypes.c_int64]),
        "gf_gnn_forward": (ctypes.c_int, [P, P, ctypes.c_int32, P, P, P, P, P]),
        "gf_gnn_loss_grad": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), P]),
        "gf_gnn_train": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
        "gf_gnn_attach": (ctypes.c_int, [P, P, ctypes.c_int32]),
        "gf_gnn_kernels_set": (ctypes.c_int, [P, ctypes.c_int32]),
        "gf_gnn_pair_get": (ctypes.c_int, [P, P, P]),
        "gf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "gf_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int) -> None:
    if status != 0:
        raise GraphFEMError(status, load_library().gf_last_error().decode())


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _arg(a, dtype, count: int, name: str):
    """(pointer, mem kind, keep-alive object) for an array argument."""
    if a is None:
        return None, None, None
    if type(a).__module__.startswith("torch"):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous {tdt} tensor")
        if a.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {a.numel()}")
        return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != count:
        raise ValueError(f"{name}: expected {count} elements, got {arr.size}")
    return arr.ctypes.data, MEM_HOST, arr


def _one_kind(*kinds) -> int:
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ks.pop() if ks else MEM_HOST


def material(young, poisson, density, threshold=math.inf, radius=0.0, alpha=0.0, beta=0.0,
             driver_mode=DRIVER_STRAIN, shear_coef=2, average_degraded=True, mass_matrix=0, energy=0) -> Material:
    """gf_material; mass_matrix MASS_LUMPED (0) or MASS_CONSISTENT (1); energy ENERGY_STVK (0) or ENERGY_SNH (1)."""
    return Material(young, poisson, density, alpha, beta, threshold, radius, driver_mode, shear_coef,
                    1 if average_degraded else 0, int(mass_matrix), int(energy), 0)


class Mesh:
    """One mesh on one GPU (opaque gf_mesh handle)."""

    def __init__(self, handle, n_nodes, n_tets, n_edges, keep):
        self._h = handle
        self.n_nodes, self.n_tets, self.n_edges = n_nodes, n_tets, n_edges
        self._keep = keep
        self._log, self._log_steps = None, 0
        _LIVE["mesh"].add(self)

    def metrics_log(self, path: Optional[str]):
        """Append one JSON line per step (step number, wall time, dt and the
        step's statistics) to `path`; None stops logging."""
        if self._log is not None:
            self._log.close()
        self._log = open(path, "a") if path else None
        self._log_steps = 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_log", None) is not None:
            self._log.close()
            self._log = None
        if self._h:
            gnn = getattr(self, "_gnn", None)
            if gnn is not None and gnn() is not None:
                gnn().close()
            load_library().gf_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> dict:
        inf = MeshInfo()
        _check(load_library().gf_mesh_info_get(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in MeshInfo._fields_}

    # -- state ------------------------------------------------------------
    def state_set(self, x=None, v=None, labels=None, chi=None):
        px, kx, kx_ = _arg(x, np.float64, 3 * self.n_nodes, "x")
        pv, kv, kv_ = _arg(v, np.float64, 3 * self.n_nodes, "v")
        pl, kl, kl_ = _arg(labels, np.uint8, self.n_edges, "labels")
        pc, kc, kc_ = _arg(chi, np.float64, self.n_tets, "chi")
        _check(load_library().gf_state_set(self._h, px, pv, pl, pc, _one_kind(kx, kv, kl, kc)))

    def step(self, dt: float, f_ext=None, pinned=None, pinned_vel=None) -> dict:
        pf, kf, kf_ = _arg(f_ext, np.float64, 3 * self.n_nodes, "f_ext")
        n_pin = 0 if pinned is None else int(np.prod(pinned.shape)) if hasattr(pinned, "shape") else len(pinned)
        pp, kp, kp_ = _arg(pinned, np.int32, n_pin, "pinned") if n_pin else (None, None, None)
        pq, kq, kq_ = _arg(pinned_vel, np.float64, 3 * n_pin, "pinned_vel") if n_pin else (None, None, None)
        st = StepStats()
        status = load_library().gf_step(self._h, float(dt), pf, pp, n_pin, pq, _one_kind(kf, kp, kq),
                                         ctypes.byref(st))
        if self._log is not None:
            self._log.write(metrics_line(self._log_steps, dt, status, st.as_dict()) + "\n")
            self._log.flush()
            self._log_steps += 1
        _check(status)
        return st.as_dict()

    def autotune(self, dt: float, f_ext=None, pinned=None, pinned_vel=None, trial_steps: int = 3):
        """gf_mesh_autotune: times the candidate schedules on the current state (restored after
        each) and keeps the fastest; returns (tuning dict, ms per step)."""
        pf, kf, kf_ = _arg(f_ext, np.float64, 3 * self.n_nodes, "f_ext")
        n_pin = 0 if pinned is None else int(np.prod(pinned.shape)) if hasattr(pinned, "shape") else len(pinned)
        pp, kp, kp_ = _arg(pinned, np.int32, n_pin, "pinned") if n_pin else (None, None, None)
        pq, kq, kq_ = _arg(pinned_vel, np.float64, 3 * n_pin, "pinned_vel") if n_pin else (None, None, None)
        best = Tuning()
        ms = ctypes.c_double(0.0)
        _check(load_library().gf_mesh_autotune(self._h, float(dt), pf, pp, n_pin, pq, _one_kind(kf, kp, kq),
                                               int(trial_steps), ctypes.byref(best), ctypes.byref(ms)))
        return {"assembly": best.assembly, "step_launch": best.step_launch, "solve_loop": best.solve_loop,
                "wait_test": best.wait_test}, ms.value

    def quasistatic_step(self, f_ext=None, pinned=None, pinned_pos=None, max_newton: int = 50,
                         rtol: float = 1e-10) -> dict:
        """gf_quasistatic_step: damage update, pinned nodes to pinned_pos, Newton with an energy line search."""
        pf, kf, kf_ = _arg(f_ext, np.float64, 3 * self.n_nodes, "f_ext")
        n_pin = 0 if pinned is None else int(np.prod(pinned.shape)) if hasattr(pinned, "shape") else len(pinned)
        pp, kp, kp_ = _arg(pinned, np.int32, n_pin, "pinned") if n_pin else (None, None, None)
        pq, kq, kq_ = _arg(pinned_pos, np.float64, 3 * n_pin, "pinned_pos") if n_pin else (None, None, None)
        st = StepStats()
        status = load_library().gf_quasistatic_step(self._h, pf, pp, n_pin, pq, _one_kind(kf, kp, kq),
                                                    int(max_newton), float(rtol), ctypes.byref(st))
        _check(status)
        return st.as_dict()

    def surface_sizes(self) -> dict:
        nv, nf, nq = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().gf_surface_sizes(self._h, ctypes.byref(nv), ctypes.byref(nf), ctypes.byref(nq)))
        return {"n_vertices": nv.value, "n_faces": nf.value, "n_quads": nq.value}

    def surface_get(self):
        """Split visualisation mesh (Sec. 4.1): vertices float64 (n, 3), crack quads int32 (q, 4)."""
        sz = self.surface_sizes()
        V = np.empty((sz["n_vertices"], 3), np.float64)
        Q = np.empty((max(sz["n_quads"], 1), 4), np.int32)
        nq = ctypes.c_int64()
        _check(load_library().gf_surface_get(self._h, V.ctypes.data, Q.ctypes.data, Q.shape[0], MEM_HOST,
                                             ctypes.byref(nq)))
        return {"vertices": V, "quads": Q[:nq.value], "n_faces": sz["n_faces"]}

    def tuning_set(self, assembly: int = None, step_launch: int = None, solve_loop: int = None,
                   wait_test: int = None):
        """gf_tuning_set; an argument left as None keeps the mesh's current value."""
        cur = self.tuning_get()
        t = Tuning()
        t.assembly = cur["assembly"] if assembly is None else assembly
        t.step_launch = cur["step_launch"] if step_launch is None else step_launch
        t.solve_loop = cur["solve_loop"] if solve_loop is None else solve_loop
        t.wait_test = cur["wait_test"] if wait_test is None else wait_test
        _check(load_library().gf_tuning_set(self._h, ctypes.byref(t)))

    def tuning_get(self) -> dict:
        t = Tuning()
        _check(load_library().gf_tuning_get(self._h, ctypes.byref(t)))
        return {"assembly": t.assembly, "step_launch": t.step_launch, "solve_loop": t.solve_loop,
                "wait_test": t.wait_test}

    def refine_set(self, inner_rtol: float):
        _check(load_library().gf_refine_set(self._h, float(inner_rtol)))

    def quasistatic_solver_set(self, solver: int, inner_rtol: float = 0.0):
        """gf_quasistatic_solver_set: QS_SOLVE_FP64 or QS_SOLVE_NESTED (inner_rtol <= 0 keeps the current one)."""
        _check(load_library().gf_quasistatic_solver_set(self._h, int(solver), float(inner_rtol)))

    def threshold_set(self, threshold: float):
        """gf_threshold_set: the break threshold of Eq. 21 between steps."""
        _check(load_library().gf_threshold_set(self._h, float(threshold)))

    def solver_set(self, rtol: float, maxit: int = 10000):
        _check(load_library().gf_solver_set(self._h, float(rtol), int(maxit)))

    def newton_set(self, max_iters: int, rtol: float = 0.0):
        """Newton iterations per step on the backward-Euler residual (FP64 meshes)."""
        _check(load_library().gf_newton_set(self._h, int(max_iters), float(rtol)))

    # -- getters ----------------------------------------------------------
    def _get(self, fn, n, dtype, out):
        if out is None:
            out = np.empty(n, dtype)
        p, k, keep = _arg(out, dtype, n, "out")
        if isinstance(out, np.ndarray) and p != out.ctypes.data:
            raise ValueError("out must be a contiguous array of the right dtype")
        _check(fn(self._h, p, k))
        return out

    def positions_get(self, out=None):
        return self._get(load_library().gf_positions_get, 3 * self.n_nodes, np.float64, out)

    def velocities_get(self, out=None):
        return self._get(load_library().gf_velocities_get, 3 * self.n_nodes, np.float64, out)

    def chi_get(self, out=None):
        return self._get(load_library().gf_chi_get, self.n_tets, np.float64, out)

    def damage_get(self):
        drv = np.empty(self.n_edges, np.float64)
        lab = np.empty(self.n_edges, np.uint8)
        _check(load_library().gf_damage_get(self._h, drv.ctypes.data, lab.ctypes.data, MEM_HOST))
        return drv, lab

    def edges_get(self):
        e = np.empty((self.n_edges, 2), np.int32)
        _check(load_library().gf_edges_get(self._h, e.ctypes.data))
        return e

    def system_get(self):
        nb = self.info["n_blocks"]
        rp = np.empty(self.n_nodes + 1, np.int32)
        col = np.empty(nb, np.int32)
        val = np.empty((nb, 3, 3), np.float64)
        rhs = np.empty(3 * self.n_nodes, np.float64)
        _check(load_library().gf_system_get(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                            rhs.ctypes.data))
        return rp, col, val, rhs

    # -- profiling --------------------------------------------------------
    def profile_enable(self, on: bool = True):
        _check(load_library().gf_profile_enable(self._h, 1 if on else 0))

    def profile_reset(self):
        _check(load_library().gf_profile_reset(self._h))

    def profile_get(self) -> dict:
        lib = load_library()
        n = 32
        ms = np.zeros(n)
        cnt = np.zeros(n, np.int64)
        k = lib.gf_profile_get(self._h, ms.ctypes.data, cnt.ctypes.data, n)
        return {lib.gf_profile_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}

    def launch_count(self) -> int:
        return int(load_library().gf_launch_count(self._h))


class Batch:
    """gf_batch: step many meshes (same device and precision) with one launch
    per kernel kind; by default each step replays one CUDA graph whose solve
    loop runs on the device."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        self.n = len(self.meshes)
        arr = (P * self.n)(*[m._h for m in self.meshes])
        h = P()
        _check(load_library().gf_batch_create(arr, self.n, ctypes.byref(h)))
        self._h = h
        _LIVE["batch"].add(self)

    def close(self):
        if getattr(self, "_h", None):
            load_library().gf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, arrays, dtype, counts, name):
        if arrays is None:
            return None, None, []
        ptrs = (P * self.n)()
        kinds, keep = [], []
        for k, a in enumerate(arrays):
            if a is None:
                continue
            p, kd, kp = _arg(a, dtype, counts[k], f"{name}[{k}]")
            ptrs[k] = p
            kinds.append(kd)
            keep.append(kp)
        return ptrs, (kinds[0] if kinds else None), keep + [ptrs]

    def _inputs(self, f_ext, pinned, pinned_vel):
        n_pin = [0] * self.n
        if pinned is not None:
            n_pin = [0 if a is None else (a.numel() if hasattr(a, "numel") else len(a)) for a in pinned]
        fp, fk, k1 = self._ptrs(f_ext, np.float64, [3 * m.n_nodes for m in self.meshes], "f_ext")
        pp, pk, k2 = self._ptrs(pinned, np.int32, n_pin, "pinned")
        vp, vk, k3 = self._ptrs(pinned_vel, np.float64, [3 * c for c in n_pin], "pinned_vel")
        npin = (ctypes.c_int64 * self.n)(*n_pin)
        mem = _one_kind(fk, pk, vk)
        return fp, pp, npin, vp, mem, k1 + k2 + k3 + [npin]

    def step(self, dt: float, f_ext=None, pinned=None, pinned_vel=None) -> list:
        fp, pp, npin, vp, mem, keep = self._inputs(f_ext, pinned, pinned_vel)
        stats = (StepStats * self.n)()
        _check(load_library().gf_batch_step(self._h, float(dt), fp, pp, npin, vp, mem, stats))
        return [st.as_dict() for st in stats]

    def tuning_set(self, graph: int = None, chunk: int = None, grid_budget: int = None, solve_loop: int = None,
                   inner: int = None):
        """gf_batch_tuning_set; an argument left as None keeps the batch's current value."""
        cur = self.tuning_get()
        t = BatchTuning()
        t.graph = cur["graph"] if graph is None else graph
        t.chunk = cur["chunk"] if chunk is None else chunk
        t.grid_budget = cur["grid_budget"] if grid_budget is None else grid_budget
        t.solve_loop = cur["solve_loop"] if solve_loop is None else solve_loop
        t.inner = cur["inner"] if inner is None else inner
        _check(load_library().gf_batch_tuning_set(self._h, ctypes.byref(t)))

    def tuning_get(self) -> dict:
        t = BatchTuning()
        _check(load_library().gf_batch_tuning_get(self._h, ctypes.byref(t)))
        return {"graph": t.graph, "chunk": t.chunk, "grid_budget": t.grid_budget, "solve_loop": t.solve_loop,
                "inner": t.inner}

    def autotune(self, dt: float, f_ext=None, pinned=None, pinned_vel=None, trial_steps: int = 3):
        fp, pp, npin, vp, mem, keep = self._inputs(f_ext, pinned, pinned_vel)
        best = BatchTuning()
        ms = ctypes.c_double(0.0)
        _check(load_library().gf_batch_autotune(self._h, float(dt), fp, pp, npin, vp, mem, int(trial_steps),
                                                ctypes.byref(best), ctypes.byref(ms)))
        return {"graph": best.graph, "chunk": best.chunk, "grid_budget": best.grid_budget, "solve_loop": best.solve_loop,
                "inner": best.inner}, ms.value

    def launch_count(self) -> int:
        return int(load_library().gf_batch_launch_count(self._h))


def mesh_plan(nodes, tets, mat: Material) -> dict:
    """gf_mesh_plan: the host precompute alone (no GPU needed)."""
    lib = load_library()
    nodes = np.ascontiguousarray(nodes, np.float64).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, np.int32).reshape(-1, 4)
    inf = MeshInfo()
    colour = np.empty(tets.shape[0], np.int32)
    cnt = np.empty(tets.shape[0], np.int32)
    _check(lib.gf_mesh_plan(nodes.ctypes.data, nodes.shape[0], tets.ctypes.data, tets.shape[0],
                            ctypes.byref(mat), ctypes.byref(inf), None, colour.ctypes.data, cnt.ctypes.data))
    edges = np.empty((inf.n_edges, 2), np.int32)
    _check(lib.gf_mesh_plan(nodes.ctypes.data, nodes.shape[0], tets.ctypes.data, tets.shape[0],
                            ctypes.byref(mat), ctypes.byref(inf), edges.ctypes.data, None, None))
    out = {f: getattr(inf, f) for f, _ in MeshInfo._fields_}
    out.update(edges=edges, colour=colour, nbr_count=cnt)
    return out


def _static_solve_args(row_ptr, col, values, b, x, fixed, device: int, stream_device):
    """Argument checks of bsr_pcg_solve_static (plain attribute access, so the
    CPU suite can run them with stand-in objects).  The C entry point launches
    on the current device with that device's scratch array, so every tensor and
    the stream must live there."""
    import torch
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col", col, torch.int32), ("values", values, torch.float64),
                        ("b", b, torch.float64), ("x", x, torch.float64), ("fixed", fixed, torch.uint8)):
        if t is None and name == "fixed":
            continue
        if not (_is_torch_cuda(t) and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name}: expected a contiguous CUDA tensor of {dt}")
        if t.device.index != device:
            raise ValueError(f"{name} lives on cuda:{t.device.index}, but the current device is cuda:{device}")
    if stream_device is not None and stream_device != device:
        raise ValueError(f"the stream belongs to cuda:{stream_device}, but the current device is cuda:{device}")
    n_rows = row_ptr.numel() - 1
    if b.numel() != 3 * n_rows or x.numel() != 3 * n_rows or (fixed is not None and fixed.numel() != n_rows):
        raise ValueError("b and x need 3 * n_rows entries, fixed n_rows")
    return n_rows


def bsr_pcg_solve_static(row_ptr, col, values, b, x, fixed=None, rtol: float = 1e-6, maxit: int = 10000,
                         stream=None):
    """gf_bsr_pcg_solve_static: solve a block-CSR system without any device
    allocation (for callers that must not allocate while solving).  All arrays
    are contiguous CUDA tensors on the current device; x holds the prescribed
    values on fixed rows (free rows are not read) and is overwritten with the
    solution.  Returns (iterations, relative residual)."""
    import torch
    device = torch.cuda.current_device()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    stream_device = stream.device.index if hasattr(stream, "device") else None
    n_rows = _static_solve_args(row_ptr, col, values, b, x, fixed, device, stream_device)
    sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    _check(load_library().gf_bsr_pcg_solve_static(row_ptr.data_ptr(), col.data_ptr(), values.data_ptr(), n_rows,
                                                  b.data_ptr(), x.data_ptr(),
                                                  None if fixed is None else fixed.data_ptr(), float(rtol),
                                                  int(maxit), sptr, ctypes.byref(it), ctypes.byref(rel)))
    return it.value, rel.value


def _torch_plumbing(device: int, stream):
    """Allocator callbacks over torch's caching allocator and the stream to use."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free), sptr


def mesh_create(nodes, tets, mat: Material, precision: int = FP64, cg_rtol: float = 1e-6, cg_maxit: int = 10000,
                device: Optional[int] = None, stream=None, torch_allocator: bool = True) -> Mesh:
    """gf_mesh_create: nodes (n,3) float64 host, tets (t,4) int32 host."""
    lib = load_library()
    nodes = np.ascontiguousarray(nodes, np.float64).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, np.int32).reshape(-1, 4)
    opt = Options()
    opt.precision = precision
    opt.cg_maxit = cg_maxit
    opt.cg_rtol = cg_rtol
    opt.precond = 0
    keep = []
    try:
        import torch
        have_torch = torch.cuda.is_available()
    except Exception:
        have_torch = False
    if device is None:
        device = torch.cuda.current_device() if have_torch else -1
    opt.device = device
    if have_torch and torch_allocator:
        a, f, sptr = _torch_plumbing(device, stream)
        opt.alloc, opt.free, opt.stream = a, f, sptr
        keep += [a, f]
    elif stream is not None:
        opt.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    h = P()
    _check(lib.gf_mesh_create(nodes.ctypes.data, nodes.shape[0], tets.ctypes.data, tets.shape[0],
                              ctypes.byref(mat), ctypes.byref(opt), ctypes.byref(h)))
    inf = MeshInfo()
    _check(lib.gf_mesh_info_get(h, ctypes.byref(inf)))
    return Mesh(h, inf.n_nodes, inf.n_tets, inf.n_edges, keep)


GNN_START, GNN_PRECOND = 1, 2
MASS_LUMPED, MASS_CONSISTENT = 0, 1
ENERGY_STVK, ENERGY_SNH = 0, 1
GNN_TENSOR_CORES, GNN_FP32_FMA = 0, 1

# Parameter tensors of the learned start / preconditioner network, in storage
# order, each row-major [in][out] (the layout gf_gnn_params_set expects).
GNN_PARAM_SHAPES = ([("W0", (16, 64)), ("b0", (64,))]
                    + [t for l in range(3) for t in ((f"Wa{l}", (64, 64)), (f"We{l}", (16, 64)), (f"bm{l}", (64,)),
                                                     (f"Wu{l}", (128, 64)), (f"bu{l}", (64,)))]
                    + [("Wd", (64, 9)), ("bd", (9,))])


class Gnn:
    """gf_gnn: learned warm start and block preconditioner for the solve of a
    GF_FP64 mesh (message passing over the mesh graph, bfloat16 weights)."""

    def __init__(self, mesh: Mesh, params=None):
        lib = load_library()
        h = P()
        _check(lib.gf_gnn_create(mesh._h, ctypes.byref(h)))
        self._h = h
        self.mesh = mesh
        mesh._gnn = weakref.ref(self)
        _LIVE["gnn"].add(self)
        self.n_params = int(lib.gf_gnn_n_params())
        self.n_graph_edges = mesh.info["n_blocks"] - mesh.n_nodes
        if params is not None:
            self.params_set(params)

    def close(self):
        if getattr(self, "_h", None):
            load_library().gf_gnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params_set(self, w):
        w = np.ascontiguousarray(w, np.float32).ravel()
        if w.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {w.size}")
        _check(load_library().gf_gnn_params_set(self._h, w.ctypes.data, w.size))

    def params_get(self) -> np.ndarray:
        w = np.empty(self.n_params, np.float32)
        _check(load_library().gf_gnn_params_get(self._h, w.ctypes.data, w.size))
        return w

    def forward(self, b) -> dict:
        """Network outputs on the mesh's last assembled system for right-hand side b."""
        n, e = self.mesh.n_nodes, self.n_graph_edges
        pb, kb, kb_ = _arg(b, np.float64, 3 * n, "b")
        out = np.empty((n, 9), np.float32)
        Pm = np.empty((n, 3, 3), np.float32)
        x0 = np.empty((n, 3), np.float32)
        fin = np.empty((n, 16), np.float32)
        ein = np.empty((max(e, 1), 16), np.float32)
        _check(load_library().gf_gnn_forward(self._h, pb, kb, out.ctypes.data, Pm.ctypes.data, x0.ctypes.data,
                                             fin.ctypes.data, ein.ctypes.data))
        return {"out": out, "P": Pm, "x0": x0, "node_in": fin, "edge_in": ein[:e]}

    def loss_grad(self, b, target):
        n = self.mesh.n_nodes
        pb, kb, kb_ = _arg(b, np.float64, 3 * n, "b")
        pt, kt, kt_ = _arg(target, np.float64, 3 * n, "target")
        loss = ctypes.c_double()
        grad = np.empty(self.n_params, np.float32)
        _check(load_library().gf_gnn_loss_grad(self._h, pb, pt, _one_kind(kb, kt), ctypes.byref(loss),
                                               grad.ctypes.data))
        return float(loss.value), grad

    def train(self, iters: int = 1, lr: float = 1e-3):
        """Adam steps on the mesh's last solved step; returns (first loss, last loss)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load_library().gf_gnn_train(self._h, int(iters), float(lr), ctypes.byref(a), ctypes.byref(b)))
        return float(a.value), float(b.value)

    def pair_get(self):
        """(b, target) of the mesh's last solved step, as gf_gnn_train uses them."""
        b = np.empty(3 * self.mesh.n_nodes)
        t = np.empty(3 * self.mesh.n_nodes)
        _check(load_library().gf_gnn_pair_get(self._h, b.ctypes.data, t.ctypes.data))
        return b, t

    def kernels_set(self, kernels: int):
        """GNN_TENSOR_CORES (tcgen05 dense contractions, default) or GNN_FP32_FMA."""
        _check(load_library().gf_gnn_kernels_set(self._h, int(kernels)))

    def attach(self, flags: int = 1):
        """GNN_START (learned start), GNN_PRECOND (learned blocks), both, or 0 (off)."""
        _check(load_library().gf_gnn_attach(self.mesh._h, self._h, int(flags)))

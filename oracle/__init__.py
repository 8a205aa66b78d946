"""FP64 CPU oracle of the SPH continuum terrain step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does, and this package imports nothing from it.

The arithmetic lives in ``crm_oracle.c`` (plain C, FP64, OpenMP over
particles); this module builds it with gcc and marshals numpy arrays.  The
simulation loop (:func:`run`) follows Alg. 2 and Alg. 3 of the paper: rebuild
the neighbour lists when the step index is a multiple of ps_freq, and, past
t_delay, refresh the activity flags at those same rebuild steps.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile crm_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (force or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("rho0", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("mu_s", C.c_double), ("mu_2", C.c_double), ("I0", C.c_double),
                ("grain_d", C.c_double), ("cohesion", C.c_double),
                ("d0", C.c_double), ("h", C.c_double),
                ("av_mode", C.c_int), ("av_gamma", C.c_double), ("av_xi2_over_h2", C.c_double),
                ("gravity", C.c_double * 3), ("kernel", C.c_int)]


def make_params(p: dict) -> Params:
    q = Params()
    for k in ("rho0", "E", "nu", "mu_s", "mu_2", "I0", "grain_d", "cohesion", "d0", "h",
              "av_gamma", "av_xi2_over_h2"):
        setattr(q, k, float(p[k]))
    q.av_mode = int(p["av_mode"])
    for k in range(3):
        q.gravity[k] = float(p["gravity"][k])
    q.kernel = int(p.get("kernel", 0))
    return q


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i64, i32, u8 = (np.ctypeslib.ndpointer(np.float64, flags="C"),
                               np.ctypeslib.ndpointer(np.int64, flags="C"),
                               np.ctypeslib.ndpointer(np.int32, flags="C"),
                               np.ctypeslib.ndpointer(np.uint8, flags="C"))
            vp = C.c_void_p
            L.orc_kernel_w.restype = C.c_double
            L.orc_kernel_w.argtypes = [C.c_double, C.c_double]
            L.orc_kernel_dwdr.restype = C.c_double
            L.orc_kernel_dwdr.argtypes = [C.c_double, C.c_double]
            L.orc_kernel_eval.argtypes = [C.c_int, C.c_double, C.c_double, d]
            L.orc_marker_kinematics.argtypes = [C.c_int64, i32, d, d, d, d, C.c_double, d, d, d]
            for nm in ("orc_neighbors_brute", "orc_neighbors_cells"):
                f = getattr(L, nm)
                f.restype = C.c_int64
                f.argtypes = [C.c_int64, C.c_int64, d, C.c_double, vp, C.c_int64, i64, i32]
            L.orc_bce.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, d, d, d, d, d, d, d,
                                  i64, i32, vp, d, d]
            L.orc_rates.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, d, d, d, d, d, d, d,
                                    i64, i32, vp, d, d, d, d, vp, vp]
            L.orc_set_scale_conditioning.argtypes = [C.c_int]
            L.orc_return_map.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, d, d, d]
            L.orc_activity.argtypes = [C.POINTER(Params), C.c_int64, d, C.c_int64, i32, d, d, d, u8]
            L.orc_capacity_policy.restype = C.c_int64
            L.orc_capacity_policy.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double,
                                              C.c_double, C.c_int64]
            L.orc_step.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, d, d, d, d,
                                   C.c_int64, i32, d, C.c_int64, d, d, d, i32, d, d, i64, i32,
                                   vp, vp, d, d]
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops (its OpenMP runtime's setting);
    returns the previous maximum."""
    L = lib()
    prev = int(L.omp_get_max_threads())
    L.omp_set_num_threads(C.c_int(int(n)))
    return prev


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def kernel_w(r: float, h: float) -> float:
    return lib().orc_kernel_w(float(r), float(h))


def kernel_dwdr(r: float, h: float) -> float:
    return lib().orc_kernel_dwdr(float(r), float(h))


KERNEL_CUBIC, KERNEL_WENDLAND = 0, 1


def kernel_eval(kind: int, r: float, h: float):
    """(W, dW/dr) of kernel `kind` (0 cubic spline, 1 quintic Wendland)."""
    out = np.zeros(2)
    lib().orc_kernel_eval(int(kind), float(r), float(h), out)
    return float(out[0]), float(out[1])


def neighbors(x_all: np.ndarray, nf: int, h: float, mode: str = "cells",
              include: Optional[np.ndarray] = None, cap: Optional[int] = None
              ) -> Tuple[np.ndarray, np.ndarray]:
    """CSR neighbour lists (offset[n+1], list[nnz]) over fluid 0..nf-1 then markers."""
    x_all = _c(x_all).reshape(-1, 3)
    n = x_all.shape[0]
    inc = None if include is None else _c(include, np.uint8)
    cap = cap if cap is not None else max(1024, 128 * n)
    off = np.zeros(n + 1, np.int64)
    lst = np.zeros(cap, np.int32)
    f = lib().orc_neighbors_brute if mode == "brute" else lib().orc_neighbors_cells
    nnz = f(nf, n - nf, x_all, float(h), _ptr(inc), cap, off, lst)
    if nnz < 0:
        raise RuntimeError("oracle neighbour capacity exceeded")
    return off, lst[:nnz].copy()


class Bodies:
    """Flat FP64 body arrays in the oracle's layout."""

    def __init__(self, scene):
        nb = len(scene.bodies)
        self.n = nb
        self.pose = np.zeros((max(nb, 1), 7))
        self.twist = np.zeros((max(nb, 1), 6))
        self.mass = np.ones(max(nb, 1))
        self.dof = np.zeros(max(nb, 1), np.int32)
        self.acc = np.zeros((max(nb, 1), 6))       # linear, angular acceleration
        self.wrench = np.zeros((max(nb, 1), 6))
        self.inertia = np.ones((max(nb, 1), 3))     # principal moments, body frame
        self.load = np.zeros((max(nb, 1), 6))       # external force, torque
        for b, body in enumerate(scene.bodies):
            self.pose[b] = body.pose
            self.twist[b] = body.twist
            self.mass[b] = body.mass
            self.dof[b] = body.dof_mask
            if getattr(body, "inertia", None) is not None:
                self.inertia[b] = body.inertia
            if getattr(body, "load", None) is not None:
                self.load[b] = body.load


def marker_arrays(scene) -> Tuple[np.ndarray, np.ndarray]:
    """(body index per marker, local coordinates) -- fixed walls first (body -1),
    then each body's markers in order."""
    parts_b = [np.full(scene.fixed.shape[0], -1, np.int32)]
    parts_x = [scene.fixed]
    for b, body in enumerate(scene.bodies):
        parts_b.append(np.full(body.markers_local.shape[0], b, np.int32))
        parts_x.append(body.markers_local)
    return _c(np.concatenate(parts_b), np.int32), _c(np.concatenate(parts_x, axis=0))


def marker_kinematics(mbody, mxloc, bodies: Bodies, tau: float):
    nm = mbody.shape[0]
    xm, um, am = np.zeros((nm, 3)), np.zeros((nm, 3)), np.zeros((nm, 3))
    lib().orc_marker_kinematics(nm, mbody, mxloc, _c(bodies.pose), _c(bodies.twist),
                                _c(bodies.acc), float(tau), xm, um, am)
    return xm, um, am


def bce(params: dict, x, u, sig, rho, xm, umb, amb, off, lst, include=None):
    nf, nm = x.shape[0], xm.shape[0]
    um, sm = np.zeros((nm, 3)), np.zeros((nm, 6))
    inc = None if include is None else _c(include, np.uint8)
    P = make_params(params)
    lib().orc_bce(C.byref(P), nf, nm, _c(x), _c(u), _c(sig), _c(rho), _c(xm) if nm else np.zeros(3),
                  _c(umb) if nm else np.zeros(3), _c(amb) if nm else np.zeros(3),
                  _c(off, np.int64), _c(lst, np.int32) if lst.size else np.zeros(1, np.int32),
                  _ptr(inc), um if nm else np.zeros(3), sm if nm else np.zeros(6))
    return um, sm


def rates(params: dict, x, u, sig, rho, xm, um, sm, off, lst, integrate=None,
          want_scale: bool = False):
    """Fluid rates (drho, du, dsig), marker accelerations and optional |term| sums
    (fluid: 10 per particle; markers: 3 per marker, returned as ``mscale``)."""
    nf, nm = x.shape[0], xm.shape[0]
    drho, du, dsig = np.zeros(nf), np.zeros((nf, 3)), np.zeros((nf, 6))
    macc = np.zeros((max(nm, 1), 3))
    scale = np.zeros((nf, 10)) if want_scale else None
    mscale = np.zeros((max(nm, 1), 3)) if want_scale else None
    ig = None if integrate is None else _c(integrate, np.uint8)
    P = make_params(params)
    z3 = np.zeros((1, 3))
    lib().orc_rates(C.byref(P), nf, nm, _c(x), _c(u), _c(sig), _c(rho),
                    _c(xm) if nm else z3, _c(um) if nm else z3, _c(sm) if nm else np.zeros((1, 6)),
                    _c(off, np.int64), _c(lst, np.int32) if lst.size else np.zeros(1, np.int32),
                    _ptr(ig), drho, du, dsig, macc, _ptr(scale), _ptr(mscale))
    return drho, du, dsig, macc[:nm], scale, (None if mscale is None else mscale[:nm])


def set_scale_conditioning(on: bool):
    """Weight the |term| sums returned with the rates by 1 + kappa(q) (kernel-edge
    conditioning); affects only the scale outputs, never a rate."""
    lib().orc_set_scale_conditioning(int(bool(on)))


def return_map(params: dict, dt: float, sig_star: np.ndarray, sig_n: Optional[np.ndarray] = None):
    s = _c(sig_star).reshape(-1, 6)
    sn = s if sig_n is None else _c(sig_n).reshape(-1, 6)
    out = np.zeros_like(s)
    P = make_params(params)
    lib().orc_return_map(C.byref(P), float(dt), s.shape[0], s, sn, out)
    return out


def activity(params: dict, x: np.ndarray, scene_boxes, pose: np.ndarray) -> np.ndarray:
    x = _c(x).reshape(-1, 3)
    nbox = len(scene_boxes)
    flag = np.zeros(x.shape[0], np.uint8)
    if nbox == 0:
        return flag
    bb = _c([b.body for b in scene_boxes], np.int32)
    bh = _c(np.stack([b.half_extents for b in scene_boxes]))
    bo = _c(np.stack([b.offset for b in scene_boxes]))
    P = make_params(params)
    lib().orc_activity(C.byref(P), x.shape[0], x, nbox, bb, bh, bo, _c(pose), flag)
    return flag


def capacity_policy(need: int, cap: int, step: int, G: float = 1.2, S: float = 0.75,
                    SI: int = 50) -> int:
    return int(lib().orc_capacity_policy(int(need), int(cap), int(step), float(G), float(S), int(SI)))


class State:
    """Mutable FP64 simulation state of one scene for the oracle loop."""

    def __init__(self, scene):
        self.scene = scene
        self.params = dict(scene.params)
        self.x = _c(scene.x).copy()
        self.u = _c(scene.u).copy()
        self.sig = _c(scene.sig).copy()
        self.rho = _c(scene.rho).copy()
        self.mbody, self.mxloc = marker_arrays(scene)
        self.bodies = Bodies(scene)
        self.step_index = 0
        self.time = 0.0          # accumulated step by step, as a time integrator does
        self.off = None
        self.lst = None
        self.include = None
        self.integrate = None
        self.flags = None
        self.marker_flags = None

    @property
    def nf(self) -> int:
        return self.x.shape[0]

    @property
    def nm(self) -> int:
        return self.mbody.shape[0]

    def markers_now(self):
        return marker_kinematics(self.mbody, self.mxloc, self.bodies, 0.0)

    def rebuild(self, mode: str = "cells"):
        """Alg. 3 items 1-4 at the current time: activity flags (past t_delay, when
        the scene has active boxes) and the neighbour lists."""
        sc = self.scene
        t = self.time
        xm, _, _ = self.markers_now()
        if sc.boxes and t > sc.t_delay:
            # Sec. 3.2 reading for markers: a body's markers always take part;
            # fixed markers take part when inside a box grown by 2h.
            self.flags = activity(self.params, self.x, sc.boxes, self.bodies.pose)
            self.marker_flags = activity(self.params, xm, sc.boxes, self.bodies.pose)
            mk = (self.marker_flags > 0) | (self.mbody >= 0)
            self.include = np.concatenate([self.flags > 0, mk]).astype(np.uint8)
            self.integrate = (self.flags == 2).astype(np.uint8)
        else:
            self.flags = None
            self.include = None
            self.integrate = None
        x_all = np.concatenate([self.x, xm], axis=0)
        self.off, self.lst = neighbors(x_all, self.nf, self.params["h"], mode, self.include)

    def step(self, dt: Optional[float] = None, mode: str = "cells"):
        """One step of Alg. 2 / Alg. 3."""
        dt = self.scene.dt if dt is None else dt
        ps = int(self.params.get("ps_freq", 1))
        if self.off is None or self.step_index % ps == 0:
            self.rebuild(mode)
        P = make_params(self.params)
        b = self.bodies
        lst = self.lst if self.lst.size else np.zeros(1, np.int32)
        lib().orc_step(C.byref(P), float(dt), self.nf, self.x, self.u, self.sig, self.rho,
                       self.nm, self.mbody if self.nm else np.zeros(1, np.int32),
                       self.mxloc if self.nm else np.zeros((1, 3)), b.n, b.pose, b.twist,
                       b.mass, b.dof, b.acc, b.wrench, self.off, lst,
                       _ptr(self.integrate), _ptr(self.include), b.inertia, b.load)
        self.step_index += 1
        self.time += dt

    def run(self, n_steps: int, dt: Optional[float] = None, mode: str = "cells"):
        for _ in range(n_steps):
            self.step(dt, mode)
        return self

    def eval_rates(self, want_scale: bool = True, mode: str = "cells"):
        """f(y) at the current state (stage-1 evaluation), without advancing."""
        self.rebuild(mode)
        xm, umb, amb = self.markers_now()
        um, sm = bce(self.params, self.x, self.u, self.sig, self.rho, xm, umb, amb,
                     self.off, self.lst, self.include)
        drho, du, dsig, macc, scale, mscale = rates(
            self.params, self.x, self.u, self.sig, self.rho, xm, um, sm, self.off, self.lst,
            self.integrate, want_scale)
        self.mscale = mscale   # |term| sums of the marker accelerations (want_scale only)
        return drho, du, dsig, macc, scale, um, sm


def run(scene, n_steps: Optional[int] = None, mode: str = "cells") -> State:
    st = State(scene)
    st.run(scene.n_steps if n_steps is None else n_steps, mode=mode)
    return st

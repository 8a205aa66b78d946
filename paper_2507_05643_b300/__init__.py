"""Python binding of the sm_103a SPH continuum terrain library (libcrm.so).

Argument marshalling only: every step of the particle loop runs in the CUDA
kernels behind the C ABI of ``include/crm.h``.  If the compiled library is
missing, importing this package raises ImportError -- there is no fallback.

Names follow the C ABI: :class:`Terrain` wraps ``crm_terrain``;
:func:`bin_points` wraps the stateless ``crm_bin_points``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2507_05643_b300/build.py` "
                      "(the CUDA library is required; there is no CPU path)")

_lib = C.CDLL(LIB_PATH)

CRM_OK = 0
STATUS = {0: "CRM_OK", -1: "CRM_EINVAL", -2: "CRM_ENOMEM", -3: "CRM_ECAPACITY",
          -4: "CRM_EESCAPED", -5: "CRM_ENONFINITE", -6: "CRM_ETIMEOUT", -7: "CRM_ECUDA",
          -8: "CRM_ESTATE"}
AV_NONE, AV_BILATERAL, AV_UNILATERAL = 0, 1, 2
DOF_X, DOF_Y, DOF_Z, DOF_RX, DOF_RY, DOF_RZ = 1, 2, 4, 8, 16, 32
KERNEL_CUBIC, KERNEL_WENDLAND = 0, 1
# parameter gradients of the reverse sweep, in this order
GRAD_NAMES = ("E", "nu", "rho0", "mu_s", "cohesion", "av_gamma", "mu_2", "I0", "grain_d")
NUM_GRADS = len(GRAD_NAMES)
# per-body gradient entries: centre, velocity, acceleration, orientation (world-frame
# rotation vector), angular velocity, angular acceleration
BODY_GRADS = 18


class CrmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("rho0", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("mu_s", C.c_double), ("mu_2", C.c_double), ("I0", C.c_double),
                ("grain_d", C.c_double), ("cohesion", C.c_double),
                ("d0", C.c_double), ("h", C.c_double),
                ("kernel", C.c_int32), ("av_mode", C.c_int32),
                ("av_gamma", C.c_double), ("av_xi2_over_h2", C.c_double),
                ("gravity", C.c_double * 3),
                ("ps_freq", C.c_int32), ("max_neighbors", C.c_int32),
                ("domain_min", C.c_double * 3), ("domain_max", C.c_double * 3),
                ("growth", C.c_double), ("shrink_ratio", C.c_double),
                ("shrink_interval", C.c_int32), ("pair_lanes", C.c_int32),
                ("skin", C.c_double)]


_d = np.ctypeslib.ndpointer(np.float64, flags="C")
_f = np.ctypeslib.ndpointer(np.float32, flags="C")
_vp, _i64, _i32 = C.c_void_p, C.c_int64, C.c_int32
_P = C.POINTER(Params)
_T = C.c_void_p


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("crm_version", C.c_int, [])
_sig("crm_status_string", C.c_char_p, [C.c_int])
_sig("crm_default_params", None, [_P])
_sig("crm_create", C.c_int, [_P, _vp, C.POINTER(_T)])
_sig("crm_destroy", C.c_int, [_T])
_sig("crm_last_error", C.c_char_p, [_T])
_sig("crm_add_sph", C.c_int, [_T, _i64, _vp, _vp, _vp, _vp])
_sig("crm_add_fixed_bce", C.c_int, [_T, _i64, _vp])
_sig("crm_add_rigid_body", C.c_int, [_T, _i64, _vp, _vp, _vp, C.c_double, _i32,
                                     C.POINTER(_i32)])
_sig("crm_set_body_motion", C.c_int, [_T, _i32, _vp, _vp])
_sig("crm_get_body_state", C.c_int, [_T, _i32, _vp, _vp])
_sig("crm_set_body_inertia", C.c_int, [_T, _i32, _vp])
_sig("crm_set_pair_lanes", C.c_int, [_T, _i32])
_sig("crm_set_cell_tile", C.c_int, [_T, _i32, _i32, _i32])
_sig("crm_debug_wait_fault", C.c_int, [_i32])
_sig("crm_debug_absolute_fp32", C.c_int, [_T, _i32])
_B = C.c_void_p
_sig("crm_batch_create", C.c_int, [_i32, C.POINTER(_T), _vp, C.POINTER(_B)])
_sig("crm_batch_step", C.c_int, [_B, _vp, _i32])
_sig("crm_batch_autotune", C.c_int, [_B, _vp, _i32, _vp])
_sig("crm_batch_destroy", C.c_int, [_B])
_sig("crm_batch_set_persistent", C.c_int, [_B, _i32])
_sig("crm_set_body_load", C.c_int, [_T, _i32, _vp, _vp])
_sig("crm_add_active_box", C.c_int, [_T, _i32, _vp, _vp, C.c_double])
_sig("crm_step", C.c_int, [_T, C.c_double, _i32])
_sig("crm_sync", C.c_int, [_T])
_sig("crm_get_particles", C.c_int, [_T, _i64, _vp, _vp, _vp, _vp, C.POINTER(_i64)])
_sig("crm_get_body_wrench", C.c_int, [_T, _i32, _vp, _vp])
_sig("crm_get_diagnostics", C.c_int, [_T, _vp])
_sig("crm_get_counts", C.c_int, [_T, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)])
_sig("crm_eval_rates", C.c_int, [_T, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp])
_sig("crm_get_neighbors", C.c_int, [_T, _i64, _vp, _vp, C.POINTER(_i64)])
_sig("crm_cosim_step", C.c_int, [_T, _vp, _vp, C.c_double, _i32, _vp, _vp, _vp])
_sig("crm_eval_rates_vjp", C.c_int, [_T, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp])
_sig("crm_adjoint_forward", C.c_int, [_T, C.c_double, _i64, _i32, _vp, _vp])
_sig("crm_adjoint_backward", C.c_int, [_T, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                       _vp, _vp])
_sig("crm_state_bytes", C.c_int, [_T, C.POINTER(C.c_size_t)])
_sig("crm_save_state", C.c_int, [_T, _vp, C.c_size_t, C.POINTER(C.c_size_t)])
_sig("crm_load_state", C.c_int, [_T, _vp, C.c_size_t])
_sig("crm_bin_scratch_bytes", C.c_size_t, [_i64, _i64])
_sig("crm_bin_points", C.c_int, [_vp, _i64, C.c_float, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp])

NUM_KERNELS = 12


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * NUM_KERNELS), ("ms", C.c_double * NUM_KERNELS),
                ("steps", C.c_int64), ("rebuilds", C.c_int64)]


_sig("crm_kernel_name", C.c_char_p, [_i32])
_sig("crm_profile_reset", C.c_int, [_T, _i32])
_sig("crm_profile_read", C.c_int, [_T, C.POINTER(Profile)])
KERNEL_NAMES = tuple(_lib.crm_kernel_name(k).decode() for k in range(NUM_KERNELS))

# Every symbol include/crm.h declares.
EXPORTS = ("crm_version", "crm_status_string", "crm_default_params", "crm_create", "crm_destroy",
           "crm_last_error", "crm_add_sph", "crm_add_fixed_bce", "crm_add_rigid_body",
           "crm_set_body_motion", "crm_get_body_state", "crm_set_body_inertia",
           "crm_set_body_load", "crm_add_active_box", "crm_step", "crm_set_pair_lanes", "crm_set_cell_tile",
           "crm_debug_wait_fault", "crm_debug_absolute_fp32",
           "crm_batch_create", "crm_batch_step", "crm_batch_autotune", "crm_batch_destroy",
           "crm_batch_set_persistent",
           "crm_sync", "crm_get_particles", "crm_get_body_wrench", "crm_get_diagnostics", "crm_get_counts",
           "crm_eval_rates", "crm_get_neighbors", "crm_state_bytes", "crm_save_state",
           "crm_load_state", "crm_bin_scratch_bytes", "crm_bin_points", "crm_kernel_name",
           "crm_profile_reset", "crm_profile_read", "crm_bin_points_noalloc",
           "crm_capacity_policy", "crm_cosim_step", "crm_eval_rates_vjp", "crm_adjoint_forward",
           "crm_adjoint_backward")


_sig("crm_capacity_policy", C.c_int, [_i64, _i64, _i64, C.c_double, C.c_double, _i32,
                                      C.POINTER(_i64)])


def capacity_policy(need: int, cap: int, step: int, growth: float = 1.2,
                    shrink_ratio: float = 0.75, shrink_interval: int = 50) -> int:
    """crm_capacity_policy: the active-set capacity after one ManageArrayMemory call."""
    out = _i64()
    rc = _lib.crm_capacity_policy(int(need), int(cap), int(step), float(growth),
                                  float(shrink_ratio), int(shrink_interval), C.byref(out))
    if rc != CRM_OK:
        raise CrmError(rc, "crm_capacity_policy rejected its arguments")
    return int(out.value)


def lib():
    return _lib


def version() -> int:
    return int(_lib.crm_version())


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64_rows(a, n: int, k: int):
    """a as a C-contiguous float64 (n, k) array (itself when it already is one)."""
    if a is None:
        return None
    if type(a) is np.ndarray and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n * k:
        return a
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(n, k))


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def default_params() -> Params:
    p = Params()
    _lib.crm_default_params(C.byref(p))
    return p


def params_from_dict(d: dict, domain_min, domain_max) -> Params:
    """crm_params from a scene's parameter dictionary and grid extent."""
    p = default_params()
    for k in ("rho0", "E", "nu", "mu_s", "mu_2", "I0", "grain_d", "cohesion", "d0", "h",
              "av_gamma", "av_xi2_over_h2", "skin"):
        if k in d and d[k] is not None:
            setattr(p, k, float(d[k]))
    for k in ("av_mode", "ps_freq", "max_neighbors", "kernel"):
        if k in d:
            setattr(p, k, int(d[k]))
    for k in range(3):
        p.gravity[k] = float(d["gravity"][k])
        p.domain_min[k] = float(domain_min[k])
        p.domain_max[k] = float(domain_max[k])
    return p


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


class Terrain:
    """Owner of one ``crm_terrain`` handle."""

    def __init__(self, params: Params, stream=None):
        self._h = _T()
        self._stream = stream
        rc = _lib.crm_create(C.byref(params), _stream_handle(stream), C.byref(self._h))
        if rc != CRM_OK:
            raise CrmError(rc, "crm_create rejected the parameters")
        self.params = params
        self.n_sph = 0
        self.n_markers = 0
        self.n_bodies = 0
        self._addrs = {}

    # ------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != CRM_OK:
            msg = _lib.crm_last_error(self._h)
            raise CrmError(rc, msg.decode() if msg else "")

    def close(self):
        if self._h:
            _lib.crm_destroy(self._h)
            self._h = _T()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def add_sph(self, xyz, vel=None, stress6=None, rho=None):
        xyz = _c(xyz).reshape(-1, 3)
        n = xyz.shape[0]
        arrs = [None if a is None else _c(a) for a in (vel, stress6, rho)]
        self._check(_lib.crm_add_sph(self._h, n, _ptr(xyz), *[_ptr(a) for a in arrs]))
        self.n_sph += n

    def add_fixed_bce(self, xyz):
        xyz = _c(xyz).reshape(-1, 3)
        self._check(_lib.crm_add_fixed_bce(self._h, xyz.shape[0], _ptr(xyz)))
        self.n_markers += xyz.shape[0]

    def add_rigid_body(self, markers_local, pose, twist, mass: float, dof_mask: int) -> int:
        ml = _c(markers_local).reshape(-1, 3)
        bid = _i32()
        self._check(_lib.crm_add_rigid_body(self._h, ml.shape[0], _ptr(ml), _ptr(_c(pose)),
                                            _ptr(_c(twist)), float(mass), int(dof_mask),
                                            C.byref(bid)))
        self.n_markers += ml.shape[0]
        self.n_bodies += 1
        return int(bid.value)

    def add_active_box(self, body: int, half_extents, offset, t_delay: float = 0.0):
        self._check(_lib.crm_add_active_box(self._h, int(body), _ptr(_c(half_extents)),
                                            _ptr(_c(offset)), float(t_delay)))

    def set_body_motion(self, body: int, pose, twist):
        self._check(_lib.crm_set_body_motion(self._h, int(body), _ptr(_c(pose)), _ptr(_c(twist))))

    def set_pair_lanes(self, lanes: int):
        self._check(_lib.crm_set_pair_lanes(self._h, int(lanes)))

    def debug_absolute_fp32(self, on: bool = True):
        """Store positions as absolute FP32 coordinates would be (the comparison
        layout of the precision tests); before the first step."""
        self._check(_lib.crm_debug_absolute_fp32(self._h, int(bool(on))))

    def set_cell_tile(self, nx: int, ny: int, nz: int):
        self._check(_lib.crm_set_cell_tile(self._h, int(nx), int(ny), int(nz)))

    def set_body_inertia(self, body: int, inertia):
        self._check(_lib.crm_set_body_inertia(self._h, int(body), _ptr(_c(inertia))))

    def set_body_load(self, body: int, force, torque):
        self._check(_lib.crm_set_body_load(self._h, int(body), _ptr(_c(force)), _ptr(_c(torque))))

    def body_state(self, body: int) -> Tuple[np.ndarray, np.ndarray]:
        pose, twist = np.zeros(7), np.zeros(6)
        self._check(_lib.crm_get_body_state(self._h, int(body), _ptr(pose), _ptr(twist)))
        return pose, twist

    # ------------------------------------------------------------------
    def step(self, dt: float, n_steps: int = 1):
        self._check(_lib.crm_step(self._h, float(dt), int(n_steps)))

    def sync(self):
        self._check(_lib.crm_sync(self._h))

    def particles(self):
        n = self.n_sph
        xyz, vel = np.zeros((n, 3)), np.zeros((n, 3), np.float32)
        sig, rho = np.zeros((n, 6), np.float32), np.zeros(n, np.float32)
        nout = _i64()
        self._check(_lib.crm_get_particles(self._h, n, _ptr(xyz), _ptr(vel), _ptr(sig), _ptr(rho),
                                           C.byref(nout)))
        return xyz, vel, sig, rho

    def cosim_step(self, dt: float, n_steps: int = 1, pose=None, twist=None, out=None):
        """One co-simulation exchange: optionally set every body's motion (pose
        (n_bodies, 7), twist (n_bodies, 6)), step, and return (wrench
        (n_bodies, 6), pose, twist) with one synchronisation.  `out`: optional
        (wrench, pose, twist) float64 arrays of those shapes to fill (no
        allocation per call)."""
        nb = self.n_bodies
        pin, tin = _f64_rows(pose, nb, 7), _f64_rows(twist, nb, 6)
        if out is None:
            out = (np.zeros((nb, 6)), np.zeros((nb, 7)), np.zeros((nb, 6)))
        w, q, v = out
        for a, k in ((w, 6), (q, 7), (v, 6)):
            if not (type(a) is np.ndarray and a.dtype == np.float64 and a.flags.c_contiguous
                    and a.size == nb * k):
                raise ValueError("cosim_step: out holds C-contiguous float64 arrays of "
                                 "(n_bodies, 6), (n_bodies, 7), (n_bodies, 6)")
        ad = self._addr
        rc = _lib.crm_cosim_step(self._h, ad(pin), ad(tin), dt, n_steps, ad(w), ad(q), ad(v))
        if rc != CRM_OK:
            self._check(rc)
        return w, q, v

    def _addr(self, a):
        """Data address of array a (None for None), remembered for the arrays a
        caller passes at every exchange."""
        if a is None:
            return None
        c = self._addrs.get(id(a))
        if c is not None and c[0] is a:
            return c[1]
        if len(self._addrs) > 16:
            self._addrs.clear()
        addr = a.ctypes.data
        self._addrs[id(a)] = (a, addr)
        return addr

    def body_wrench(self, body: int) -> Tuple[np.ndarray, np.ndarray]:
        f, t = np.zeros(3), np.zeros(3)
        self._check(_lib.crm_get_body_wrench(self._h, int(body), _ptr(f), _ptr(t)))
        return f, t

    def diagnostics(self) -> dict:
        """FP64 global sums over the SPH particles (crm_get_diagnostics): count,
        mass, volume, momentum (3), angular momentum about the origin (3), kinetic
        energy."""
        out = np.zeros(10)
        self._check(_lib.crm_get_diagnostics(self._h, _ptr(out)))
        return {"count": out[0], "mass": out[1], "volume": out[2], "momentum": out[3:6].copy(),
                "angular_momentum": out[6:9].copy(), "kinetic_energy": out[9]}

    def counts(self) -> Tuple[int, int, int]:
        a, e, b = _i64(), _i64(), _i64()
        self._check(_lib.crm_get_counts(self._h, C.byref(a), C.byref(e), C.byref(b)))
        return int(a.value), int(e.value), int(b.value)

    def eval_rates(self):
        """(drho, du, dsig, marker_acc, marker_vel, marker_sig) at the current state."""
        n, m = self.n_sph, self.n_markers
        drho, du, ds = np.zeros(n, np.float32), np.zeros((n, 3), np.float32), np.zeros((n, 6), np.float32)
        ma, mv, ms = (np.zeros((m, 3), np.float32), np.zeros((m, 3), np.float32),
                      np.zeros((m, 6), np.float32))
        self._check(_lib.crm_eval_rates(self._h, n, _ptr(drho), _ptr(du), _ptr(ds), m, _ptr(ma),
                                        _ptr(mv), _ptr(ms)))
        return drho, du, ds, ma, mv, ms

    def _grads(self, call) -> dict:
        n, nb = self.n_sph, self.n_bodies
        out = {"params": np.zeros(NUM_GRADS), "xyz": np.zeros((n, 3)), "vel": np.zeros((n, 3)),
               "stress": np.zeros((n, 6)), "rho": np.zeros(n), "body": np.zeros((max(nb, 1), BODY_GRADS))}
        self._check(call(out))
        out["body"] = out["body"][:nb]
        out["param_grads"] = dict(zip(GRAD_NAMES, (float(v) for v in out["params"])))
        return out

    def eval_rates_vjp(self, l_drho=None, l_dvel=None, l_dstress=None, l_macc=None) -> dict:
        """Gradient of sum(l . rates of eval_rates) at the current state (each l
        optional): {'xyz', 'vel', 'stress', 'rho' (per SPH particle), 'body'
        (per body: centre, velocity, acceleration, orientation as a world-frame
        rotation vector, angular velocity, angular acceleration), 'params'
        (GRAD_NAMES order),
        'param_grads' (by name)}."""
        n, m = self.n_sph, self.n_markers

        def arr(a, shape):
            return None if a is None else np.ascontiguousarray(np.asarray(a, np.float32).reshape(shape))
        ld, lu, ls, lm = arr(l_drho, (n,)), arr(l_dvel, (n, 3)), arr(l_dstress, (n, 6)), arr(l_macc, (m, 3))
        return self._grads(lambda o: _lib.crm_eval_rates_vjp(
            self._h, n, _ptr(ld), _ptr(lu), _ptr(ls), m, _ptr(lm), _ptr(o["xyz"]), _ptr(o["vel"]),
            _ptr(o["stress"]), _ptr(o["rho"]), _ptr(o["body"]), _ptr(o["params"])))

    def adjoint_forward(self, dt: float, n_steps: int, every: int) -> Tuple[np.ndarray, np.ndarray]:
        """Run n_steps steps with checkpoints every `every` steps; returns the soil
        wrench (n_steps, n_bodies, 6) and the pose (n_steps, n_bodies, 7) after
        each step."""
        nb = self.n_bodies
        w = np.zeros((n_steps, max(nb, 1), 6))
        q = np.zeros((n_steps, max(nb, 1), 7))
        self._check(_lib.crm_adjoint_forward(self._h, float(dt), int(n_steps), int(every),
                                             _ptr(w), _ptr(q)))
        return w[:, :nb], q[:, :nb]

    def adjoint_backward(self, l_wrench=None, l_center=None, l_xyz=None, l_vel=None,
                         l_stress=None, l_rho=None) -> dict:
        """Gradient of an objective of the recorded run given dJ/d wrench
        (n_steps, n_bodies, 6), dJ/d centre after each step (n_steps, n_bodies,
        3) and dJ/d final SPH state (l_xyz, l_vel (n, 3), l_stress (n, 6), l_rho
        (n,)): parameters and the initial state, as eval_rates_vjp."""
        def arr(a):
            return None if a is None else np.ascontiguousarray(np.asarray(a, np.float64))
        lw, lc, lx, lu, ls, lr = (arr(a) for a in (l_wrench, l_center, l_xyz, l_vel, l_stress, l_rho))
        return self._grads(lambda o: _lib.crm_adjoint_backward(
            self._h, _ptr(lw), _ptr(lc), _ptr(lx), _ptr(lu), _ptr(ls), _ptr(lr), _ptr(o["params"]),
            _ptr(o["xyz"]), _ptr(o["vel"]), _ptr(o["stress"]), _ptr(o["rho"]), _ptr(o["body"])))

    def neighbors(self) -> Tuple[np.ndarray, np.ndarray]:
        n = self.n_sph + self.n_markers
        off = np.zeros(n + 1, np.int64)
        nnz = _i64()
        self._check(_lib.crm_get_neighbors(self._h, 0, _ptr(off), None, C.byref(nnz)))
        lst = np.zeros(max(int(nnz.value), 1), np.int32)
        self._check(_lib.crm_get_neighbors(self._h, lst.size, _ptr(off), _ptr(lst), C.byref(nnz)))
        return off, lst[:int(nnz.value)]

    def profile_reset(self, timing: bool = False):
        self._check(_lib.crm_profile_reset(self._h, int(bool(timing))))

    def profile(self) -> dict:
        """{'launches': {name: n}, 'ms': {name: ms}, 'steps': n, 'rebuilds': n}."""
        pr = Profile()
        self._check(_lib.crm_profile_read(self._h, C.byref(pr)))
        return {"launches": {KERNEL_NAMES[k]: int(pr.launches[k]) for k in range(NUM_KERNELS)},
                "ms": {KERNEL_NAMES[k]: float(pr.ms[k]) for k in range(NUM_KERNELS)},
                "steps": int(pr.steps), "rebuilds": int(pr.rebuilds)}

    def state_bytes(self) -> int:
        b = C.c_size_t()
        self._check(_lib.crm_state_bytes(self._h, C.byref(b)))
        return int(b.value)

    def save_state(self, dev_ptr: int, cap: int) -> int:
        used = C.c_size_t()
        self._check(_lib.crm_save_state(self._h, C.c_void_p(dev_ptr), cap, C.byref(used)))
        return int(used.value)

    def load_state(self, dev_ptr: int, used: int):
        self._check(_lib.crm_load_state(self._h, C.c_void_p(dev_ptr), used))


def from_scene(scene, stream=None, **param_over) -> Terrain:
    """Terrain holding a ``scenes.Scene``: its SPH particles, fixed walls, bodies
    and active boxes, with the scene's constants (overridable by keyword)."""
    d = dict(scene.params)
    d.update(param_over)
    t = Terrain(params_from_dict(d, scene.domain_min, scene.domain_max), stream)
    t.add_sph(scene.x, scene.u, scene.sig, scene.rho)
    if scene.fixed.shape[0]:
        t.add_fixed_bce(scene.fixed)
    for k, b in enumerate(scene.bodies):
        t.add_rigid_body(b.markers_local, b.pose, b.twist, b.mass, b.dof_mask)
        if getattr(b, "inertia", None) is not None:
            t.set_body_inertia(k, b.inertia)
        if getattr(b, "load", None) is not None:
            t.set_body_load(k, b.load[:3], b.load[3:])
    for bx in scene.boxes:
        t.add_active_box(bx.body, bx.half_extents, bx.offset, scene.t_delay)
    return t


class Batch:
    """``crm_batch`` over Terrain members, each created with its own stream: one
    call steps every member concurrently (the members stay owned by the caller)."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        arr = (_T * len(self.members))(*[m._h.value for m in self.members])
        self._b = _B()
        rc = _lib.crm_batch_create(len(self.members), arr, _stream_handle(stream),
                                   C.byref(self._b))
        if rc != CRM_OK:
            raise CrmError(rc, "crm_batch_create: members need distinct handles, each on a stream")

    def _dts(self, dt):
        return _c(np.broadcast_to(np.asarray(dt, np.float64), (len(self.members),)))

    def step(self, dt, n_steps: int = 1):
        rc = _lib.crm_batch_step(self._b, _ptr(self._dts(dt)), int(n_steps))
        if rc != CRM_OK:
            raise CrmError(rc, "crm_batch_step failed (see the members' last errors)")

    def set_persistent(self, on: bool = True):
        """Step the batch by one graph with one persistent launch per stage over
        all members (on), or by the members' own graphs on their streams (off)."""
        rc = _lib.crm_batch_set_persistent(self._b, int(bool(on)))
        if rc != CRM_OK:
            raise CrmError(rc, "crm_batch_set_persistent failed")

    def autotune(self, dt, trial_steps: int = 3) -> np.ndarray:
        choice = np.zeros(len(self.members), np.int32)
        rc = _lib.crm_batch_autotune(self._b, _ptr(self._dts(dt)), int(trial_steps),
                                     choice.ctypes.data_as(C.c_void_p))
        if rc != CRM_OK:
            raise CrmError(rc, "crm_batch_autotune failed")
        return choice

    def close(self):
        if self._b:
            _lib.crm_batch_destroy(self._b)
            self._b = _B()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bin_points(xyz_ptr: int, n: int, cell_size: float, dims, cell_ptr: int, perm_ptr: int,
               start_ptr: int, scratch_ptr: int, scratch_bytes: int, stream=None):
    """crm_bin_points on device pointers (e.g. torch tensors' data_ptr())."""
    d = (C.c_int32 * 3)(*[int(v) for v in dims])
    rc = _lib.crm_bin_points(C.c_void_p(xyz_ptr), int(n), float(cell_size), d,
                             C.c_void_p(cell_ptr), C.c_void_p(perm_ptr), C.c_void_p(start_ptr),
                             C.c_void_p(scratch_ptr), int(scratch_bytes),
                             _stream_handle(stream))
    if rc != CRM_OK:
        raise CrmError(rc, "crm_bin_points rejected its arguments")


_sig("crm_bin_points_noalloc", C.c_int, [_vp, _i64, C.c_float, _vp, _vp, _vp, _vp, _vp])


def bin_points_noalloc(xyz_ptr: int, n: int, cell_size: float, dims, cell_ptr: int,
                       perm_ptr: int, start_ptr: int, stream=None):
    """crm_bin_points_noalloc on device pointers: the same binning with the
    library's built-in scratch array (for callers that cannot allocate)."""
    d = (C.c_int32 * 3)(*[int(v) for v in dims])
    rc = _lib.crm_bin_points_noalloc(C.c_void_p(xyz_ptr), int(n), float(cell_size), d,
                                     C.c_void_p(cell_ptr), C.c_void_p(perm_ptr),
                                     C.c_void_p(start_ptr), _stream_handle(stream))
    if rc != CRM_OK:
        raise CrmError(rc, "crm_bin_points_noalloc rejected its arguments")


def debug_wait_fault(on: bool):
    """crm_debug_wait_fault: make the device waits of the look-back scans on the
    current device run out (on) or behave normally (off) -- a test hook."""
    rc = _lib.crm_debug_wait_fault(int(bool(on)))
    if rc != CRM_OK:
        raise CrmError(rc, "crm_debug_wait_fault failed")


def bin_scratch_bytes(n: int, ncell: int) -> int:
    return int(_lib.crm_bin_scratch_bytes(int(n), int(ncell)))

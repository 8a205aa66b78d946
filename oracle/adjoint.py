"""The oracle's own FP64 adjoint -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the benchmark's CPU legs may import this module; the
product path never does.

The step of ``crm_oracle.c`` (two-stage midpoint integration of Sec. 2.2 with
the BCE boundary of Sec. 2.4, the return map of Sec. 2.3 and the rigid-body
update) is restated here with plain PyTorch CPU tensor operations in float64,
one pass over all pairs of the oracle's CSR neighbour lists per sum, and
differentiated by reverse-mode automatic differentiation.  The readings are
those of the C oracle (the artificial-viscosity sign, c_s = sqrt(K / rho0),
marker density rho0, Adami's stress extrapolation, the ghost velocity
2 u_body - u~, the return map applied once to sigma* at the end of the step,
I = 0 when the shear rate or p* is not positive, Euler's equations with the
world-frame inertia at t_n).

Neighbour lists are built by the C oracle from each step's start positions and
held fixed through the step, as in the C oracle; the derivative is the one of
the run with those lists, on the branches (unilateral viscosity, return-map
case, mu(I)) the run takes.  The run is reversed one step at a time: the
forward keeps each step's start state; the backward re-evaluates a step under
autograd from its start state and pulls the incoming adjoint through it.

This module shares no code with the CUDA path and none of its arithmetic with
``crm_oracle.c`` (it imports the C oracle only for the neighbour lists and the
scene's marker arrays).  ``tests/test_oracle_adjoint.py`` pins it to the C
oracle: the forward step to rounding, the gradients to FP64 central
differences of the C oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np
import torch

from . import Bodies, marker_arrays, neighbors

# Differentiable material constants (the C ABI's gradient order).
PARAMS = ("E", "nu", "rho0", "mu_s", "cohesion", "av_gamma", "mu_2", "I0", "grain_d")

_F64 = torch.float64


def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=_F64)


# ---------------------------------------------------------------------------
# Kernels (Sec. 3.1): W(r) and dW/dr with support 2h.
def _kernel(kind: int, r: torch.Tensor, h: float):
    q = r / h
    if kind == 1:   # Wendland C2 of radius 2h: 21/(16 pi h^3) (1 - q/2)^4 (2q + 1)
        a = 21.0 / (16.0 * math.pi * h ** 3)
        t = torch.clamp(1.0 - 0.5 * q, min=0.0)
        W = a * t ** 4 * (2.0 * q + 1.0)
        dW = -5.0 * a / h * q * t ** 3
        return W, dW
    # cubic M4 spline, 1 / (pi h^3)
    s = 1.0 / (math.pi * h ** 3)
    t = torch.clamp(2.0 - q, min=0.0)
    inner = q < 1.0
    W = torch.where(inner, s * (1.0 - 1.5 * q * q + 0.75 * q ** 3), s * 0.25 * t ** 3)
    dW = torch.where(inner, s / h * (-3.0 * q + 2.25 * q * q), -0.75 * s / h * t * t)
    return W, dW


# ---------------------------------------------------------------------------
# Quaternions (w, x, y, z) and rigid kinematics.
def _qmul(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([aw * bw - ax * bx - ay * by - az * bz,
                        aw * bx + ax * bw + ay * bz - az * by,
                        aw * by - ax * bz + ay * bw + az * bx,
                        aw * bz + ax * by - ay * bx + az * bw], -1)


def _rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of a unit quaternion (the map v -> q v q*)."""
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _advance(q: torch.Tensor, w: torch.Tensor, tau: float) -> torch.Tensor:
    """exp(tau w / 2) q, normalised: the turn by the rotation vector tau w.
    cos(a) and sin(a) / a with a^2 = tau^2 |w|^2 / 4 are taken as functions of
    a^2 (a series below 1e-4, so that a rate of zero has a finite derivative)."""
    x = (w * w).sum(-1) * (0.25 * tau * tau)
    small = x < 1e-4
    xs = torch.where(small, torch.ones_like(x), x)
    a = torch.sqrt(xs)
    c = torch.where(small, 1 - x / 2 * (1 - x / 12 * (1 - x / 30)), torch.cos(a))
    sa = torch.where(small, 1 - x / 6 * (1 - x / 20 * (1 - x / 42)), torch.sin(a) / a)
    dq = torch.cat([c.unsqueeze(-1), (0.5 * tau * sa).unsqueeze(-1) * w], -1)
    o = _qmul(dq, q)
    return o / torch.sqrt((o * o).sum(-1, keepdim=True))


@dataclass
class BodyState:
    """Per-body tensors: pose (nb, 7), twist (nb, 6), accelerations (nb, 6)."""
    pose: torch.Tensor
    twist: torch.Tensor
    acc: torch.Tensor


def _marker_kin(mbody: np.ndarray, mxloc: torch.Tensor, B: BodyState, tau: float):
    """Marker positions, rigid velocities and accelerations at stage offset tau
    (fixed markers: their world position, at rest)."""
    nm = mbody.shape[0]
    xm = mxloc.clone()
    um = torch.zeros((nm, 3), dtype=_F64)
    am = torch.zeros((nm, 3), dtype=_F64)
    if nm == 0 or B.pose.shape[0] == 0:
        return xm, um, am
    on = torch.as_tensor(mbody >= 0)
    if not bool(on.any()):
        return xm, um, am
    idx = torch.as_tensor(np.where(mbody >= 0, mbody, 0).astype(np.int64))
    xc = B.pose[:, :3] + tau * B.twist[:, :3]
    q = _advance(B.pose[:, 3:], B.twist[:, 3:], tau)
    R = _rotmat(q)[idx]                                   # (nm, 3, 3)
    rl = torch.einsum("aij,aj->ai", R, mxloc)
    w = B.twist[idx, 3:]
    al = B.acc[idx, 3:]
    wr = torch.cross(w, rl, dim=-1)
    xb = xc[idx] + rl
    ub = B.twist[idx, :3] + wr
    ab = B.acc[idx, :3] + torch.cross(al, rl, dim=-1) + torch.cross(w, wr, dim=-1)
    m = on.unsqueeze(-1)
    return torch.where(m, xb, xm), torch.where(m, ub, um), torch.where(m, ab, am)


# ---------------------------------------------------------------------------
@dataclass
class Pairs:
    """CSR lists as pair arrays: row i, column j (flat index: fluid, then markers)."""
    i: torch.Tensor
    j: torch.Tensor
    n: int

    @staticmethod
    def from_csr(off: np.ndarray, lst: np.ndarray) -> "Pairs":
        n = off.shape[0] - 1
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
        return Pairs(torch.as_tensor(rows), torch.as_tensor(lst.astype(np.int64)), n)


def _sum_rows(n: int, rows: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    out = torch.zeros((n,) + tuple(v.shape[1:]), dtype=_F64)
    return out.index_add(0, rows, v)


def _full(s6: torch.Tensor) -> torch.Tensor:
    xx, yy, zz, xy, xz, yz = s6.unbind(-1)
    return torch.stack([torch.stack([xx, xy, xz], -1), torch.stack([xy, yy, yz], -1),
                        torch.stack([xz, yz, zz], -1)], -2)


def _bce(P: dict, kind: int, nf: int, pr: Pairs, xf, uf, sf, rf, xm, umb, amb, grav):
    """Marker velocity and stress (Sec. 2.4, Adami extrapolation in stress form):
    over each marker's fluid neighbours f, w = sum W, u~ = sum u_f W / w,
    u_a = 2 u_body - u~, sigma_a = [sum sigma_f W - ((g - a_a) . sum rho_f (x_a - x_f) W) I] / w;
    u_a = u_body and sigma_a = 0 without fluid in reach."""
    nm = xm.shape[0]
    sel = pr.i >= nf
    a = pr.i[sel] - nf
    f = pr.j[sel]
    d = xm[a] - xf[f]
    W, _ = _kernel(kind, torch.sqrt((d * d).sum(-1)), P["h"])
    w = _sum_rows(nm, a, W)
    su = _sum_rows(nm, a, uf[f] * W[:, None])
    ss = _sum_rows(nm, a, sf[f] * W[:, None])
    sr = _sum_rows(nm, a, (rf[f] * W)[:, None] * d)
    has = w > 0.0
    ws = torch.where(has, w, torch.ones_like(w))
    gp = ((grav[None, :] - amb) * sr).sum(-1)
    um = torch.where(has[:, None], 2.0 * umb - su / ws[:, None], umb)
    iso = torch.tensor([1.0, 1.0, 1.0, 0.0, 0.0, 0.0], dtype=_F64)
    sm = torch.where(has[:, None], (ss - gp[:, None] * iso[None, :]) / ws[:, None],
                     torch.zeros_like(ss))
    return um, sm


def _rates(P: dict, M: dict, kind: int, av_mode: int, nf: int, pr: Pairs,
           xf, uf, sf, rf, xm, um, sm):
    """Rates of the fluid (F2 continuity and velocity gradient, F3 momentum with
    viscosity and gravity, Jaumann stress rate) and the marker accelerations
    (momentum sum without gravity), Sec. 2.1-2.2 and 2.4."""
    h = P["h"]
    X = torch.cat([xf, xm], 0)
    U = torch.cat([uf, um], 0)
    S = torch.cat([sf, sm], 0)
    Rh = torch.cat([rf, M["rho0"].expand(xm.shape[0])], 0)
    i, j = pr.i, pr.j
    rij = X[i] - X[j]
    r = torch.sqrt((rij * rij).sum(-1))
    _, dW = _kernel(kind, r, h)
    g = (dW / r)[:, None] * rij                       # grad_i W_ij (no pair has r = 0)
    Vj = M["m"] / Rh[j]
    uji = U[j] - U[i]
    Ssum = _full(S[i]) + _full(S[j])
    mom = _sum_rows(pr.n, i, Vj[:, None] * torch.einsum("pab,pb->pa", Ssum, g))
    if av_mode != 0:
        vr = -(uji * rij).sum(-1)
        rbar = 0.5 * (Rh[i] + Rh[j])
        fac = (M["av_gamma"] * h * (M["m"] / rbar) * M["cs"] * vr
               / ((rij * rij).sum(-1) + P["av_xi2_over_h2"] * h * h))
        if av_mode == 2:
            fac = torch.where(vr < 0.0, fac, torch.zeros_like(fac))
        av = _sum_rows(pr.n, i, fac[:, None] * g)
    else:
        av = torch.zeros((pr.n, 3), dtype=_F64)
    fl = i < nf
    cont = _sum_rows(pr.n, i, torch.where(fl, Vj * (uji * g).sum(-1), torch.zeros_like(Vj)))
    Lp = (Vj[:, None] * uji)[:, :, None] * g[:, None, :]
    L = _sum_rows(pr.n, i, torch.where(fl[:, None, None], Lp, torch.zeros_like(Lp)))[:nf]
    rhoi = rf
    drho = -rhoi * cont[:nf]
    grav = M["grav"]
    du = mom[:nf] / rhoi[:, None] + grav[None, :] + av[:nf]
    # stress rate: Omega sigma - sigma Omega + 2G (eps - tr/3 I) + K tr I
    E = 0.5 * (L + L.transpose(1, 2))
    Om = 0.5 * (L - L.transpose(1, 2))
    Sf = _full(sf)
    tr = E.diagonal(dim1=1, dim2=2).sum(-1)
    I3 = torch.eye(3, dtype=_F64)
    Rt = (Om @ Sf - Sf @ Om + 2.0 * M["G"] * (E - (tr / 3.0)[:, None, None] * I3)
          + (M["K"] * tr)[:, None, None] * I3)
    dsig = torch.stack([Rt[:, 0, 0], Rt[:, 1, 1], Rt[:, 2, 2], Rt[:, 0, 1], Rt[:, 0, 2],
                        Rt[:, 1, 2]], -1)
    macc = mom[nf:] / M["rho0"] + av[nf:]
    return drho, du, dsig, macc


def _taubar(s: torch.Tensor) -> torch.Tensor:
    p = -(s[:, 0] + s[:, 1] + s[:, 2]) / 3.0
    t = s[:, :3] + p[:, None]
    tt = (t * t).sum(-1) + 2.0 * (s[:, 3:] * s[:, 3:]).sum(-1)
    return torch.sqrt(torch.clamp(0.5 * tt, min=1e-300))


def _return_map(M: dict, dt: float, s: torch.Tensor, sn: torch.Tensor) -> torch.Tensor:
    """Sec. 2.3: tension cut-off, mu(I), cone test, radial return of the
    deviator (the C oracle's four steps, as masks)."""
    ps = -(s[:, 0] + s[:, 1] + s[:, 2]) / 3.0
    tb = _taubar(s)
    mu_s, mu_2, c = M["mu_s"], M["mu_2"], M["cohesion"]
    cut = (ps < -c / mu_s) if float(mu_s.detach()) > 0.0 else torch.zeros_like(ps, dtype=torch.bool)
    mu = mu_s.expand(ps.shape)
    if float(mu_2.detach()) != float(mu_s.detach()):
        gdot = (tb - _taubar(sn)) / (M["G"] * dt)
        rate = (gdot > 0.0) & (ps > 0.0)
        ps_s = torch.where(rate, ps, torch.ones_like(ps))
        gd_s = torch.where(rate, gdot, torch.ones_like(gdot))
        I = gd_s * M["grain_d"] * torch.sqrt(M["rho0"] / ps_s)
        mu = torch.where(rate, mu_s + (mu_2 - mu_s) / (1.0 + M["I0"] / I), mu)
    tmax = mu * ps + c
    keep = tb <= tmax
    f = tmax / tb
    iso = torch.tensor([1.0, 1.0, 1.0, 0.0, 0.0, 0.0], dtype=_F64)
    ret = -ps[:, None] * iso + f[:, None] * (s + ps[:, None] * iso)
    out = torch.where(keep[:, None], s, ret)
    return torch.where(cut[:, None], torch.zeros_like(s), out)


def _materials(P: dict, T: Dict[str, torch.Tensor]) -> dict:
    E, nu, rho0 = T["E"], T["nu"], T["rho0"]
    G = E / (2.0 * (1.0 + nu))
    K = E / (3.0 * (1.0 - 2.0 * nu))
    M = dict(T)
    M.update(G=G, K=K, m=rho0 * P["d0"] ** 3, cs=torch.sqrt(K / rho0),
             grav=_t(P["gravity"]))
    return M


@dataclass
class Static:
    """What a run holds fixed: constants, markers, body constants."""
    P: dict
    kind: int
    av_mode: int
    mbody: np.ndarray
    mxloc: torch.Tensor
    mass: torch.Tensor
    dof: np.ndarray
    inertia: torch.Tensor
    load: torch.Tensor
    nb: int


def step(S: Static, T: Dict[str, torch.Tensor], dt: float, x, u, sig, rho, B: BodyState,
         pr: Pairs):
    """One step of the C oracle's orc_step on tensors (lists `pr` fixed).
    Returns (x, u, sig, rho, bodies after the step, wrench (nb, 6))."""
    P = S.P
    M = _materials(P, T)
    nf = x.shape[0]
    grav = M["grav"]
    # stage 1 at y_n
    xm, umb, amb = _marker_kin(S.mbody, S.mxloc, B, 0.0)
    um, sm = _bce(P, S.kind, nf, pr, x, u, sig, rho, xm, umb, amb, grav)
    d1, du1, ds1, _ = _rates(P, M, S.kind, S.av_mode, nf, pr, x, u, sig, rho, xm, um, sm)
    hd = 0.5 * dt
    xh, uh, sh, rh = x + hd * u, u + hd * du1, sig + hd * ds1, rho + hd * d1
    # stage 2 at the midpoint
    xm, umb, amb = _marker_kin(S.mbody, S.mxloc, B, 0.5 * dt)
    um, sm = _bce(P, S.kind, nf, pr, xh, uh, sh, rh, xm, umb, amb, grav)
    d2, du2, ds2, macc = _rates(P, M, S.kind, S.av_mode, nf, pr, xh, uh, sh, rh, xm, um, sm)
    x1 = x + dt * uh
    u1 = u + dt * du2
    r1 = rho + dt * d2
    s1 = _return_map(M, dt, sig + dt * ds2, sig)
    # wrench at the midpoint configuration
    nb = S.nb
    wrench = torch.zeros((nb, 6), dtype=_F64)
    if nb:
        onb = S.mbody >= 0
        a_idx = torch.as_tensor(np.nonzero(onb)[0].astype(np.int64))
        b_idx = torch.as_tensor(S.mbody[onb].astype(np.int64))
        xc = B.pose[:, :3] + 0.5 * dt * B.twist[:, :3]
        f = M["m"] * macc[a_idx]
        rr = xm[a_idx] - xc[b_idx]
        F = _sum_rows(nb, b_idx, f)
        Tq = _sum_rows(nb, b_idx, torch.cross(rr, f, dim=-1))
        wrench = torch.cat([F, Tq], -1)
    # body update: symplectic Euler of the free DOFs
    pose, twist, acc = [], [], []
    for b in range(nb):
        Fb = wrench[b, :3] + S.load[b, :3]
        Tb = wrench[b, 3:] + S.load[b, 3:]
        dof = int(S.dof[b])
        w = B.twist[b, 3:]
        wdot = torch.zeros(3, dtype=_F64)
        if dof & (7 << 3):
            R = _rotmat(B.pose[b, 3:])
            Iw = R @ torch.diag(S.inertia[b]) @ R.T
            rhs = Tb - torch.cross(w, Iw @ w, dim=-1)
            wdot = R @ ((R.T @ rhs) / S.inertia[b])
        lin = [Fb[c] / S.mass[b] + grav[c] if dof & (1 << c) else None for c in range(3)]
        v_new = torch.stack([B.twist[b, c] + dt * lin[c] if lin[c] is not None else B.twist[b, c]
                             for c in range(3)])
        w_new = torch.stack([w[c] + dt * wdot[c] if dof & (8 << c) else w[c] for c in range(3)])
        a_new = torch.stack([lin[c] if lin[c] is not None else torch.zeros((), dtype=_F64)
                             for c in range(3)]
                            + [wdot[c] if dof & (8 << c) else torch.zeros((), dtype=_F64)
                               for c in range(3)])
        c_new = B.pose[b, :3] + dt * v_new
        q_new = _advance(B.pose[b, 3:], w_new, dt)
        pose.append(torch.cat([c_new, q_new]))
        twist.append(torch.cat([v_new, w_new]))
        acc.append(a_new)
    if nb:
        B1 = BodyState(torch.stack(pose), torch.stack(twist), torch.stack(acc))
    else:
        B1 = BodyState(B.pose, B.twist, B.acc)
    return x1, u1, s1, r1, B1, wrench


# ---------------------------------------------------------------------------
def static_of(scene) -> Static:
    mbody, mxloc = marker_arrays(scene)
    bd = Bodies(scene)
    nb = bd.n
    return Static(P=dict(scene.params), kind=int(scene.params.get("kernel", 0)),
                  av_mode=int(scene.params["av_mode"]), mbody=mbody, mxloc=_t(mxloc),
                  mass=_t(bd.mass[:nb]), dof=bd.dof[:nb].copy(), inertia=_t(bd.inertia[:nb]),
                  load=_t(bd.load[:nb]), nb=nb)


def _lists(S: Static, x: np.ndarray, B: BodyState, mode: str) -> Pairs:
    with torch.no_grad():
        xm, _, _ = _marker_kin(S.mbody, S.mxloc, BodyState(B.pose.detach(), B.twist.detach(),
                                                           B.acc.detach()), 0.0)
    x_all = np.concatenate([x, xm.numpy()], 0)
    off, lst = neighbors(x_all, x.shape[0], S.P["h"], mode)
    return Pairs.from_csr(off, lst)


class Run:
    """A recorded oracle run: forward() keeps each step's start state (the
    backward builds that step's lists from it again, the same lists);
    backward(...) returns the FP64 gradients of
    J = sum_s lw_s . wrench_s + lc_s . centre_s + lfin . final SPH state
    with respect to the material constants (PARAMS), the initial SPH state, and
    the bodies' initial centre, velocity, world-frame rotation vector of the
    orientation and angular velocity."""

    def __init__(self, scene, mode: Optional[str] = None):
        self.scene = scene
        self.S = static_of(scene)
        self.mode = mode or ("brute" if scene.x.shape[0] < 4000 else "cells")
        self.T0 = {k: _t(float(scene.params[k])) for k in PARAMS}
        bd = Bodies(scene)
        nb = bd.n
        self.B0 = BodyState(_t(bd.pose[:nb]), _t(bd.twist[:nb]), _t(bd.acc[:nb]))
        self.y0 = tuple(_t(a) for a in (scene.x, scene.u, scene.sig, scene.rho))
        self.tape: List[tuple] = []

    def forward(self, dt: float, n_steps: int):
        """Returns the wrench (n_steps, nb, 6) and pose (n_steps, nb, 7) after each step."""
        self.dt = dt
        self.tape = []
        x, u, sig, rho = self.y0
        B = self.B0
        W, Q = [], []
        with torch.no_grad():
            for _ in range(n_steps):
                pr = _lists(self.S, x.numpy(), B, self.mode)
                self.tape.append(((x, u, sig, rho), B))
                x, u, sig, rho, B, wr = step(self.S, self.T0, dt, x, u, sig, rho, B, pr)
                W.append(wr.numpy().copy())
                Q.append(B.pose.numpy().copy())
        self.final = (x, u, sig, rho, B)
        nb = self.S.nb
        return (np.array(W).reshape(n_steps, nb, 6), np.array(Q).reshape(n_steps, nb, 7))

    def backward(self, lw=None, lc=None, lfin: Optional[dict] = None) -> dict:
        n = len(self.tape)
        nf = self.y0[0].shape[0]
        nb = self.S.nb
        # adjoints of the state after the last step
        ly = [torch.zeros((nf, 3), dtype=_F64), torch.zeros((nf, 3), dtype=_F64),
              torch.zeros((nf, 6), dtype=_F64), torch.zeros(nf, dtype=_F64)]
        if lfin is not None:
            ly = [_t(lfin[k]).reshape(v.shape) for k, v in zip(("x", "u", "sig", "rho"), ly)]
        lB = [torch.zeros((nb, 7), dtype=_F64), torch.zeros((nb, 6), dtype=_F64),
              torch.zeros((nb, 6), dtype=_F64)]
        gT = {k: 0.0 for k in PARAMS}
        lw = None if lw is None else np.asarray(lw, dtype=np.float64).reshape(n, nb, 6)
        lc = None if lc is None else np.asarray(lc, dtype=np.float64).reshape(n, nb, 3)
        for s in reversed(range(n)):
            (x, u, sig, rho), B = self.tape[s]
            pr = _lists(self.S, x.numpy(), B, self.mode)     # the forward's lists again
            xs = [a.clone().requires_grad_(True) for a in (x, u, sig, rho)]
            Bs = BodyState(B.pose.clone().requires_grad_(True), B.twist.clone().requires_grad_(True),
                           B.acc.clone().requires_grad_(True))
            T = {k: v.clone().requires_grad_(True) for k, v in self.T0.items()}
            x1, u1, s1, r1, B1, wr = step(self.S, T, self.dt, *xs, Bs, pr)
            J = (ly[0] * x1).sum() + (ly[1] * u1).sum() + (ly[2] * s1).sum() + (ly[3] * r1).sum()
            if nb:
                lpose = lB[0].clone()
                if lc is not None:
                    lpose[:, :3] += _t(lc[s])
                J = J + (lpose * B1.pose).sum() + (lB[1] * B1.twist).sum() + (lB[2] * B1.acc).sum()
                if lw is not None:
                    J = J + (_t(lw[s]) * wr).sum()
            ins = xs + ([Bs.pose, Bs.twist, Bs.acc] if nb else []) + [T[k] for k in PARAMS]
            gr = torch.autograd.grad(J, ins, allow_unused=True)
            gr = [torch.zeros_like(a) if g is None else g for g, a in zip(gr, ins)]
            ly = list(gr[:4])
            if nb:
                lB = list(gr[4:7])
            for k, g in zip(PARAMS, gr[-len(PARAMS):]):
                gT[k] += float(g)
        out = {"x": ly[0].numpy(), "u": ly[1].numpy(), "sig": ly[2].numpy(),
               "rho": ly[3].numpy(), "params": gT}
        if nb:
            # the orientation's adjoint as the adjoint of a world-frame rotation
            # vector theta at the initial pose: q(theta) = exp(theta / 2) q0, so
            # dq / dtheta = 1/2 [0, theta] q0 at theta = 0
            q0 = self.B0.pose[:, 3:]
            lq = lB[0][:, 3:]
            lth = torch.zeros((nb, 3), dtype=_F64)
            for k in range(3):
                e = torch.zeros(4, dtype=_F64)
                e[1 + k] = 0.5
                lth[:, k] = (lq * _qmul(e.expand_as(q0), q0)).sum(-1)
            out["body_c"] = lB[0][:, :3].numpy()
            out["body_theta"] = lth.numpy()
            out["body_v"] = lB[1][:, :3].numpy()
            out["body_w"] = lB[1][:, 3:].numpy()
            out["body_acc"] = lB[2].numpy()
        return out


def run_gradients(scene, dt: float, n_steps: int, lw=None, lc=None, lfin=None,
                  mode: Optional[str] = None):
    """Forward and reverse sweep of a run; returns (wrench, pose, gradients)."""
    r = Run(scene, mode)
    w, q = r.forward(dt, n_steps)
    return w, q, r.backward(lw, lc, lfin)


def _wheel_test(n_steps: int = 400, threads: int = 0) -> dict:
    """The differentiable wheel test (30,000 SPH particles on a 1.0 x 0.3 x 0.1 m
    bin, the wheel-bin wheel and material, 5e-5 s steps): gradients of the mean
    drawbar pull F_x and of the mean sinkage z0 - z over the second half of the
    run with respect to the friction angle, cohesion, E, rho0 and the wheel's
    prescribed forward speed and spin, with the time per step of the forward and
    of each reverse sweep."""
    import json
    import time

    import scenes
    if threads:
        torch.set_num_threads(threads)
    sc = scenes.wheel_bin(seed=3, nx=100, ny=30, nz=10)
    r = Run(sc, "cells")
    t0 = time.perf_counter()
    _, q = r.forward(sc.dt, n_steps)
    t_fwd = time.perf_counter() - t0
    half = n_steps // 2
    lw = np.zeros((n_steps, 1, 6))
    lw[half:, 0, 0] = 1.0 / (n_steps - half)
    lc = np.zeros((n_steps, 1, 3))
    lc[half:, 0, 2] = -1.0 / (n_steps - half)
    mu = float(sc.params["mu_s"])
    out = {"n_sph": int(sc.x.shape[0]), "steps": n_steps, "threads": torch.get_num_threads(),
           "forward_s_per_step": t_fwd / n_steps}
    for name, (a, b) in (("drawbar_pull", (lw, None)), ("sinkage", (None, lc))):
        t0 = time.perf_counter()
        g = r.backward(a, b)
        out[name + "_backward_s_per_step"] = (time.perf_counter() - t0) / n_steps
        out[name] = {"phi": g["params"]["mu_s"] * (1.0 + mu * mu),
                     "cohesion": g["params"]["cohesion"], "E": g["params"]["E"],
                     "rho0": g["params"]["rho0"], "speed_x": float(g["body_v"][0, 0]),
                     "omega_y": float(g["body_w"][0, 1])}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    import sys
    _wheel_test(int(sys.argv[1]) if len(sys.argv) > 1 else 400)

"""The state a terrain holds, computed on the host from its definition (a test
helper; no GPU output is involved).

The library stores each particle's position as an FP32 offset from the corner of
its home cell -- cells of 2h (1 + skin) from the domain minimum, that size rounded
up to an FP32 value (2h without a skin, and with active boxes) -- and velocities,
stresses and densities as FP32 values; a body marker's position is rounded the
same way at every stage.  The FP64 oracle fed with that state sees the very
inputs the kernels see, so a parity bar on the rates measures the kernels'
arithmetic alone, not the rounding of their inputs.
"""
import numpy as np

import oracle


def cell_size(params: dict, skin: float) -> float:
    """Edge of the library's grid cells: 2h (1 + skin) rounded up to an FP32 value."""
    req = 2.0 * float(params["h"]) * (1.0 + skin)
    c = np.float32(req)
    if float(c) < req:
        c = np.nextafter(c, np.float32(np.inf))
    return float(c)


def hold_positions(x: np.ndarray, dmin, cell: float) -> np.ndarray:
    """FP64 positions rebuilt from the FP32 offsets to the home-cell corners:
    c = floor((x - dmin) / cell), x' = dmin + c cell + fp32(x - (dmin + c cell))."""
    x = np.asarray(x, np.float64)
    dm = np.asarray(dmin, np.float64)
    c = np.floor((x - dm) / cell)
    corner = dm + c * cell
    off = (x - corner).astype(np.float32).astype(np.float64)
    return corner + off


def held_scene(sc, skin: float):
    """A copy of scene `sc` with its SPH state and fixed markers as a terrain
    built from it holds them."""
    h = sc.copy()
    cell = cell_size(sc.params, skin)
    h.x = hold_positions(sc.x, sc.domain_min, cell)
    h.u = sc.u.astype(np.float32).astype(np.float64)
    h.sig = sc.sig.astype(np.float32).astype(np.float64)
    h.rho = sc.rho.astype(np.float32).astype(np.float64)
    if sc.fixed.shape[0]:
        h.fixed = hold_positions(sc.fixed, sc.domain_min, cell)
    return h


def eval_rates(st: "oracle.State", skin: float, conditioned: bool = False):
    """The oracle's rate evaluation of state `st` (built from a held scene) with
    its body markers rounded as the terrain rounds them at the current pose:
    (drho, du, dsig, macc, scale, marker_scale, um, sm)."""
    sc = st.scene
    cell = cell_size(sc.params, skin)
    xm, umb, amb = st.markers_now()
    body = st.mbody >= 0
    if np.any(body):
        xm = xm.copy()
        xm[body] = hold_positions(xm[body], sc.domain_min, cell)
    x_all = np.concatenate([st.x, xm], axis=0)
    off, lst = oracle.neighbors(x_all, st.nf, st.params["h"], "cells")
    um, sm = oracle.bce(st.params, st.x, st.u, st.sig, st.rho, xm, umb, amb, off, lst)
    oracle.set_scale_conditioning(conditioned)
    try:
        drho, du, dsig, macc, scale, mscale = oracle.rates(
            st.params, st.x, st.u, st.sig, st.rho, xm, um, sm, off, lst, None, True)
    finally:
        oracle.set_scale_conditioning(False)
    return drho, du, dsig, macc, scale, mscale, um, sm


def _kernel_edge_kappa(st, skin, h):
    """Per marker: the largest kernel-edge amplification kappa = 2q/(2-q) over its
    fluid neighbours (large when a neighbour sits right at 2h)."""
    cell = cell_size(st.params, skin)
    xm, _, _ = st.markers_now()
    body = st.mbody >= 0
    xm = xm.copy()
    xm[body] = hold_positions(xm[body], st.scene.domain_min, cell)
    x_all = np.concatenate([st.x, xm], axis=0)
    off, lst = oracle.neighbors(x_all, st.nf, h, "cells")
    kmax = np.zeros(st.nm)
    for a in range(st.nm):
        row = lst[off[st.nf + a]:off[st.nf + a + 1]]
        if row.size:
            q = np.linalg.norm(st.x[row] - xm[a], axis=1) / h
            kmax[a] = np.max(2 * q / (2 - q))
    return kmax


def check_rates(name, sc, rates, skin=0.1, edge_kappa=400.0, tol=1e-5):
    """The rate parity bars on the GPU rates `rates` (as Terrain.eval_rates returns
    them) of a terrain built from scene `sc`: every fluid component within tol S,
    every marker acceleration component within tol S or -- a marker with a
    neighbour at the kernel edge (largest kappa >= edge_kappa, kappa = 2q/(2-q)
    the factor by which W' ~ (2 - q)^2 amplifies a relative rounding of r) --
    within tol S' (the sums with each term weighted by 1 + kappa); marker
    velocity and stress within 4 tol of the largest fluid value.  Returns the
    marker components that needed the kernel-edge bar: (marker, component,
    largest kappa, err/S, err/S')."""
    drho, du, ds, macc, mvel, msig = rates
    hs = held_scene(sc, skin)
    st = oracle.State(hs)
    o_drho, o_du, o_ds, o_macc, scale, mscale, o_um, o_sm = eval_rates(st, skin)
    got = np.concatenate([drho[:, None], du, ds], axis=1).astype(np.float64)
    ref = np.concatenate([o_drho[:, None], o_du, o_ds], axis=1)
    err = np.abs(got - ref)
    worst = np.max(err / np.maximum(scale, 1e-30))
    assert np.all(err <= tol * scale + 1e-30), f"{name}: worst err/S = {worst:.3e}"
    edge = []
    if st.nm:
        merr = np.abs(macc.astype(np.float64) - o_macc)
        over = np.argwhere(merr > tol * mscale + 1e-30)
        if over.size:
            kmax = _kernel_edge_kappa(st, skin, sc.params["h"])
            *_, cscale, cmscale, _, _ = eval_rates(st, skin, conditioned=True)
            for a, c in over:
                edge.append((int(a), int(c), float(kmax[a]), float(merr[a, c] / mscale[a, c]),
                             float(merr[a, c] / cmscale[a, c])))
            print(f"{name}: kernel-edge marker components (marker, comp, max kappa, err/S, "
                  f"err/S'): {edge}")
            assert all(k >= edge_kappa and r2 <= tol for _, _, k, _, r2 in edge), edge
        umax = max(np.abs(st.u).max(), 1e-6)
        assert np.all(np.abs(mvel - o_um) <= tol * umax * 4 + 1e-7)
        smax = max(np.abs(st.sig).max(), 1.0)
        assert np.all(np.abs(msig - o_sm) <= tol * smax * 4)
    return edge

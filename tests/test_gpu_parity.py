"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (the single-precision reading of the parity tolerances):
* integer work (cells, sort order, cell ranges) is bit-exact; neighbour sets are
  exact except pairs whose FP64 distance lies within 1e-6 h of the 2h cut-off
  (an FP32 evaluation may decide those either way);
* single-step rates: |r_gpu - r_oracle| <= 1e-5 * S per particle and component,
  S = sum_j |term_ij| from the oracle (rates of a body at rest cancel to ~0, so a
  plain relative error is undefined; a momentum term's size is that of the
  products it adds, sigma_i dW and sigma_j dW), with the oracle fed the state the
  terrain holds (tests/held.py: FP32 cell-relative positions, FP32 velocity,
  stress and density) so that the bar measures the kernels' arithmetic;
* marker accelerations: the same bar; a marker component over it must be one
  of a marker with a neighbour at the kernel edge (a pair at q >= 1.99, where
  W' ~ (2 - q)^2 amplifies the FP32 rounding of r by kappa = 2q/(2-q) >= 400)
  and must meet the bar against S' = sum_j |term_ij| (1 + kappa_j) instead; the
  random-state wheel scene has 16 such components of 8 wheel markers;
* marker velocity / stress: the extrapolation is a convex weighting, so the bar
  is 1e-5 of the largest fluid value involved;
* one step: the same bars carried through the two RK2 stages (dt times twice the
  rate tolerance, plus the FP32 rounding of the stored state);
* short horizons: reported per quantity at steps 1, 10, 50, 200, with stress
  measured against the lithostatic scale rho0 g H of the column.
"""
import math

import numpy as np
import pytest

import held
import oracle
import scenes

pytestmark = pytest.mark.gpu

crm = pytest.importorskip("paper_2507_05643_b300")
RATE_TOL = 1e-5
BAND = 1e-6   # neighbour pairs within BAND * h of 2h are not compared


def _rand_state(sc, seed, u_amp=0.3, s_lo=-3000.0, s_hi=300.0):
    rng = np.random.default_rng(seed)
    sc.u = rng.uniform(-u_amp, u_amp, size=sc.u.shape)
    sc.sig = rng.uniform(s_lo, s_hi, size=sc.sig.shape)
    sc.rho = sc.params["rho0"] * (1 + rng.uniform(-0.01, 0.01, size=sc.rho.shape))
    return sc


def _scenes():
    a = _rand_state(scenes.lattice_only(seed=11, n=14, av_mode=1, av_gamma=0.3), 11)
    b = _rand_state(scenes.settling_block(seed=12, n=12, box=0.18), 12)
    c = scenes.wheel_bin(seed=13, nx=40, ny=24, nz=10, wheel_radius=0.08, wheel_width=0.08,
                         n_grousers=8, wheel_x=0.2)
    c.bodies[0].pose[2] -= 0.005    # grousers sunk into the soil
    c = _rand_state(c, 13, u_amp=0.05, s_lo=-2500, s_hi=-100)
    return {"lattice": a, "block": b, "wheel": c}


SCENES = _scenes()


@pytest.fixture(scope="module", params=sorted(SCENES))
def pair(request):
    sc = SCENES[request.param].copy()
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    return request.param, sc, t, st


def _all_positions(st):
    xm, _, _ = st.markers_now()
    return np.concatenate([st.x, xm], axis=0)


# --------------------------------------------------------------------------
def test_neighbor_sets_match_oracle(pair):
    name, sc, t, st = pair
    t.eval_rates()
    off_g, lst_g = t.neighbors()
    x = _all_positions(st)
    off_o, lst_o = oracle.neighbors(x, st.nf, sc.params["h"], "brute" if x.shape[0] < 9000 else "cells")
    h2 = 2 * sc.params["h"]
    n = x.shape[0]
    assert off_g.shape[0] == n + 1
    mism = 0
    for i in range(n):
        g = set(lst_g[off_g[i]:off_g[i + 1]].tolist())
        o = set(lst_o[off_o[i]:off_o[i + 1]].tolist())
        for j in g ^ o:
            r = np.linalg.norm(x[i] - x[j])
            if abs(r - h2) >= BAND * sc.params["h"]:
                mism += 1
    assert mism == 0
    assert lst_g.size > 20 * st.nf


def test_rates_match_oracle(pair):
    name, sc, t, st = pair
    edge = held.check_rates(name, sc, t.eval_rates())
    assert len(edge) <= 20


def test_gpu_momentum_antisymmetry():
    sc = scenes.lattice_only(seed=21, n=16, av_mode=1, av_gamma=0.5)
    sc = _rand_state(sc, 21)
    sc.params["gravity"] = (0.0, 0.0, 0.0)
    t = crm.from_scene(sc)
    _, du, *_ = t.eval_rates()
    tot = du.astype(np.float64).sum(axis=0)
    assert np.all(np.abs(tot) <= 1e-6 * np.abs(du).astype(np.float64).sum(axis=0))


def test_gpu_momentum_balance_with_markers():
    sc = _rand_state(scenes.settling_block(seed=22, n=10, box=0.16), 22)
    sc.params["gravity"] = (0.0, 0.0, 0.0)
    t = crm.from_scene(sc)
    _, du, _, macc, _, _ = t.eval_rates()
    tot = du.astype(np.float64).sum(axis=0) + macc.astype(np.float64).sum(axis=0)
    ref = np.abs(du).astype(np.float64).sum(axis=0) + np.abs(macc).astype(np.float64).sum(axis=0)
    assert np.all(np.abs(tot) <= 1e-6 * ref)


# --------------------------------------------------------------------------
def _compare_states(t, st, d0, sig_scale):
    xyz, vel, sig, rho = t.particles()
    dx = np.max(np.abs(xyz - st.x)) / d0
    du = np.sqrt(np.mean((vel - st.u) ** 2)) / max(np.sqrt(np.mean(st.u ** 2)), 1e-12)
    ds = np.sqrt(np.mean((sig - st.sig) ** 2)) / sig_scale
    dr = np.sqrt(np.mean((rho - st.rho) ** 2)) / np.sqrt(np.mean(st.rho ** 2))
    return dx, du, ds, dr


def test_single_step_elastic_matches_oracle():
    """One full step (both RK2 stages, markers moving with the wheel) with the
    return map kept inactive (cohesion 1e9): y_{n+1} within dt * 2 * 1e-5 * S of
    the oracle's step, plus FP32 rounding of the stored state."""
    sc = scenes.wheel_bin(seed=41, nx=40, ny=24, nz=10, wheel_radius=0.08, wheel_width=0.08,
                          n_grousers=8, wheel_x=0.2)
    sc.bodies[0].pose[2] -= 0.006
    sc = _rand_state(sc, 41, u_amp=0.05, s_lo=-2000, s_hi=-200)
    sc.params["cohesion"] = 1e9
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    oracle.set_scale_conditioning(True)
    try:
        *_, scale, _, _ = st.eval_rates(want_scale=True)
    finally:
        oracle.set_scale_conditioning(False)
    dt = sc.dt
    t.step(dt, 1)
    st2 = oracle.State(sc)
    st2.step()
    xyz, vel, sig, rho = t.particles()
    eps = np.finfo(np.float32).eps
    tol_u = dt * 2 * RATE_TOL * scale[:, 1:4] + 4 * eps * np.abs(st2.u) + 1e-9
    tol_s = dt * 2 * RATE_TOL * scale[:, 4:10] + 4 * eps * np.abs(st2.sig) + 1e-6
    tol_r = dt * 2 * RATE_TOL * scale[:, 0] + 4 * eps * st2.rho
    assert np.all(np.abs(vel - st2.u) <= tol_u), np.max(np.abs(vel - st2.u) / tol_u)
    assert np.all(np.abs(sig - st2.sig) <= tol_s), np.max(np.abs(sig - st2.sig) / tol_s)
    assert np.all(np.abs(rho - st2.rho) <= tol_r), np.max(np.abs(rho - st2.rho) / tol_r)
    assert np.max(np.abs(xyz - st2.x)) <= 1e-8
    F, T = t.body_wrench(0)
    Fo = st2.bodies.wrench[0, :3]
    assert np.linalg.norm(F) > 0
    assert np.linalg.norm(F - Fo) <= 1e-4 * np.linalg.norm(Fo)


def test_return_map_on_isolated_particles():
    """Particles 3h apart have no neighbours, so one step gives sigma* = sigma_n and
    the kernel returns RM(sigma_n): compare with the oracle's FP64 return map."""
    rng = np.random.default_rng(42)
    n = 12
    sc = scenes.lattice_only(seed=42, n=n, d0=0.04, jitter=0.0, random_state=False,
                             mu_s=0.55, cohesion=300.0)
    sc.params["h"] = 0.012
    sc.params["gravity"] = (0.0, 0.0, 0.0)
    m = sc.x.shape[0]
    s = rng.normal(0, 3000, size=(m, 6))
    s[:, :3] -= rng.uniform(-500, 3000, size=(m, 1))
    p_star = -(s[:, 0] + s[:, 1] + s[:, 2]) / 3
    s = s[np.abs(p_star + 300 / 0.55) > 1.0]   # keep clear of the tension cut-off
    sc.x, sc.u, sc.rho = sc.x[:s.shape[0]], sc.u[:s.shape[0]], sc.rho[:s.shape[0]]
    sc.sig = s
    t = crm.from_scene(sc)
    t.step(1e-4, 1)
    _, _, sig, _ = t.particles()
    ref = oracle.return_map(sc.params, 1e-4, s.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(sig - ref) <= 1e-5 * np.abs(s).max(axis=1, keepdims=True))
    zero = np.all(ref == 0, axis=1)
    assert zero.sum() > 10 and (~zero).sum() > 10
    assert np.all(sig[zero] == 0)


def test_settling_block_short_horizon():
    """The 8,000-particle settling block (3-layer walls, 30 deg, c = 0, bilateral
    AV 0.02, dt 1e-4) against the FP64 oracle at steps 1, 10, 50 and 200."""
    sc = scenes.settling_block()
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    d0 = sc.params["d0"]
    sig_scale = sc.params["rho0"] * 9.81 * 0.2
    done = 0
    report = {}
    for k in (1, 10, 50, 200):
        t.step(sc.dt, k - done)
        st.run(k - done)
        done = k
        report[k] = _compare_states(t, st, d0, sig_scale)
    print("settling block: max|dx|/d0, rms du/rms u, rms dsig/(rho0 g H), rms drho/rho:", report)
    dx1, du1, ds1, dr1 = report[1]
    assert dx1 < 1e-6 and ds1 < 1e-5 and dr1 < 1e-6, report
    dx, du, ds, dr = report[200]
    assert dx < 1e-3 and ds < 1e-3 and dr < 1e-5, report


def test_wheel_short_horizon_and_wrench():
    sc = scenes.wheel_bin(seed=43, nx=40, ny=24, nz=10, wheel_radius=0.08, wheel_width=0.08,
                          n_grousers=8, wheel_x=0.2)
    sc.bodies[0].pose[2] -= 0.004
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    sig_scale = sc.params["rho0"] * 9.81 * 0.1
    report = {}
    done = 0
    for k in (1, 10, 50, 100):
        t.step(sc.dt, k - done)
        st.run(k - done)
        done = k
        F, T = t.body_wrench(0)
        Fo = st.bodies.wrench[0, :3]
        report[k] = _compare_states(t, st, sc.params["d0"], sig_scale) + (
            float(np.linalg.norm(F - Fo) / max(np.linalg.norm(Fo), 1e-12)),)
    print("wheel: max|dx|/d0, rms du/rms u, rms dsig/(rho0 g H), rms drho/rho, |dF|/|F|:", report)
    assert report[1][0] < 1e-6 and report[1][4] < 1e-4, report
    dx, du, ds, dr, dF = report[100]
    assert dx < 1e-3 and ds < 1e-3 and dF < 1e-2, report
    pose, twist = t.body_state(0)
    assert abs(pose[2] - st.bodies.pose[0, 2]) < 1e-6
    assert abs(twist[2] - st.bodies.twist[0, 2]) < 1e-3 * max(1.0, abs(st.bodies.twist[0, 2]))


def test_step_is_deterministic():
    sc = scenes.settling_block(seed=31, n=12, box=0.18)
    outs = []
    for _ in range(2):
        t = crm.from_scene(sc)
        t.step(sc.dt, 25)
        outs.append(t.particles())
        t.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_checkpoint_roundtrip():
    torch = pytest.importorskip("torch")
    sc = scenes.settling_block(seed=32, n=10, box=0.16)
    t = crm.from_scene(sc)
    t.step(sc.dt, 3)
    nb = t.state_bytes()
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    used = t.save_state(buf.data_ptr(), nb)
    t.step(sc.dt, 5)
    a = t.particles()
    t.load_state(buf.data_ptr(), used)
    t.step(sc.dt, 5)
    b = t.particles()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


# --------------------------------------------------------------------------
# Failure paths: made on the host, reported as status codes, nothing faults.

def test_capacity_overflow_reported():
    sc = scenes.settling_block(seed=33, n=8, box=0.12)
    t = crm.from_scene(sc, max_neighbors=8)
    t.step(sc.dt, 1)
    with pytest.raises(crm.CrmError) as e:
        t.sync()
    assert e.value.code == -3


def test_escape_reported():
    sc = scenes.settling_block(seed=34, n=6, box=0.1)
    sc.u[0] = [0.0, 0.0, 5000.0]   # leaves the grid within a step
    t = crm.from_scene(sc)
    t.step(sc.dt, 2)
    with pytest.raises(crm.CrmError) as e:
        t.sync()
    assert e.value.code in (-4, -5)


def test_nonfinite_reported():
    sc = scenes.settling_block(seed=35, n=6, box=0.1)
    sc.sig[:] = 3.0e38
    t = crm.from_scene(sc)
    t.step(sc.dt, 1)
    with pytest.raises(crm.CrmError) as e:
        t.sync()
    assert e.value.code == -5


# --------------------------------------------------------------------------
# Stateless binning (Sec. 3.1 steps 1-3): bit-exact against its definition.

@pytest.mark.parametrize("n, dims, spread", [
    (0, (3, 2, 2), 1.0), (1, (1, 1, 1), 1.0), (4097, (9, 7, 5), 1.0),
    (250_000, (88, 22, 29), 1.0), (1_000_003, (200, 40, 30), 1.0),
    # degenerate distributions: every point in one cell; ~90 % of the points
    # outside the grid, clamped into its boundary cells; a grid whose cell index
    # needs all four 8-bit digits of the radix sort
    (200_000, (1, 1, 1), 1.0), (300_000, (64, 32, 16), 10.0), (100_000, (512, 256, 200), 1.0)])
def test_bin_points_exact(n, dims, spread):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n)
    cell = np.float32(0.024)
    ext = np.array(dims, np.float32) * cell
    xyz = ((rng.uniform(-0.01, 1.0, size=(n, 3)) - 0.5) * spread + 0.5) * ext
    xyz = xyz.astype(np.float32)
    if n > 10:
        xyz[:5] = np.float32(cell) * np.float32(2.0)   # points exactly on cell faces
    ncell = int(np.prod(dims))
    dev = torch.device("cuda")
    X = torch.from_numpy(xyz.reshape(-1)).to(dev) if n else torch.zeros(3, device=dev)
    cells = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    perm = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    start = torch.zeros(ncell + 1, dtype=torch.int32, device=dev)
    sb = crm.bin_scratch_bytes(n, ncell)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    for _ in range(2):   # twice: the scratch carries no state between calls
        crm.bin_points(X.data_ptr(), n, float(cell), dims, cells.data_ptr(), perm.data_ptr(),
                       start.data_ptr(), scratch.data_ptr(), sb)
        torch.cuda.synchronize()
    inv = np.float32(1.0) / cell
    ijk = np.floor(xyz * inv).astype(np.int64)
    ijk = np.clip(ijk, 0, np.array(dims) - 1)
    c_ref = (ijk[:, 2] * dims[1] + ijk[:, 1]) * dims[0] + ijk[:, 0]
    perm_ref = np.argsort(c_ref, kind="stable")
    start_ref = np.searchsorted(c_ref[perm_ref], np.arange(ncell + 1), side="left")
    assert np.array_equal(cells.cpu().numpy()[:n].astype(np.int64), c_ref)
    assert np.array_equal(perm.cpu().numpy()[:n].astype(np.int64), perm_ref)
    assert np.array_equal(start.cpu().numpy().astype(np.int64), start_ref)


# --------------------------------------------------------------------------
# Verlet skin: the exact 2h lists filtered from skin lists equal a fresh search

@pytest.mark.parametrize("skin", [0.0, 0.1, 0.3])
def test_skin_lists_stay_exact_over_many_steps(skin):
    sc = _rand_state(scenes.settling_block(seed=61, n=12, box=0.18), 61, u_amp=0.6)
    t = crm.from_scene(sc, skin=skin)
    t.profile_reset()
    n = 45
    t.step(sc.dt, n)
    t.eval_rates()                      # a rebuild at the current positions
    prof = t.profile()
    off_g, lst_g = t.neighbors()
    xyz, *_ = t.particles()
    st = oracle.State(sc)
    xm, _, _ = st.markers_now()
    x = np.concatenate([xyz, xm], axis=0)
    off_o, lst_o = oracle.neighbors(x, sc.n_fluid, sc.params["h"], "cells")
    h = sc.params["h"]
    bad = 0
    for i in range(x.shape[0]):
        for j in set(lst_g[off_g[i]:off_g[i + 1]].tolist()) ^ set(lst_o[off_o[i]:off_o[i + 1]].tolist()):
            if abs(np.linalg.norm(x[i] - x[j]) - 2 * h) >= BAND * h:
                bad += 1
    assert bad == 0
    searches = prof["launches"]["neighbors"]
    if skin > 0:
        assert 2 <= searches < prof["rebuilds"], prof   # the skin saves searches but does some
    else:
        assert searches == prof["rebuilds"], prof


@pytest.mark.parametrize("skin", [0.0, 0.1])
def test_settling_block_skin_variants_agree(skin):
    """Same trajectory with and without the skin (identical neighbour sets; only
    the summation order of the pairs differs)."""
    sc = scenes.settling_block(seed=62, n=14, box=0.2)
    a = crm.from_scene(sc, skin=skin)
    a.step(sc.dt, 60)
    b = crm.from_scene(sc, skin=0.0)
    b.step(sc.dt, 60)
    xa, _, sa, _ = a.particles()
    xb, _, sb, _ = b.particles()
    # FP32 rounding only: offsets from cells of 2h (1 + skin) vs 2h, other pair order
    assert np.max(np.abs(xa - xb)) < 1e-5 * sc.params["d0"]
    assert np.sqrt(np.mean((sa - sb) ** 2)) < 1e-5 * sc.params["rho0"] * 9.81 * 0.14

"""The reverse sweep (hand-derived adjoint) against central differences of the
FP64 oracle.

Each check is a directional derivative: for a random direction d of one input
group, <g, d> from the adjoint must match (J(y + e d) - J(y - e d)) / 2e of the
oracle, J = sum(l . outputs) with random weights l.  The oracle's neighbour
lists are built once at the base point (the adjoint differentiates with the
lists held fixed), and the state is chosen so that no branch (the unilateral
viscosity switch, the return map's cases) sits within the difference step.
Bar: |<g, d> - FD| <= TOL * sum_i |g_i d_i| (the sum of the magnitudes of the
dot product's terms: the adjoint is FP32 arithmetic, the difference FP64).
"""
import copy

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

crm = pytest.importorskip("paper_2507_05643_b300")
TOL = 2e-3          # rate evaluation
RUN_TOL = 1e-2      # a run of steps (FP32 trajectory against the FP64 one)


def _wheel(seed=21, nx=24, ny=16, nz=8):
    sc = scenes.wheel_bin(seed=seed, nx=nx, ny=ny, nz=nz, wheel_radius=0.06, wheel_width=0.06,
                          n_grousers=8, wheel_x=0.12)
    sc.bodies[0].pose[2] -= 0.004   # grousers in the soil
    rng = np.random.default_rng(seed)
    sc.u = rng.uniform(-0.05, 0.05, size=sc.u.shape)
    sc.sig = sc.sig + rng.uniform(-300.0, 300.0, size=sc.sig.shape)
    sc.rho = sc.params["rho0"] * (1 + rng.uniform(-0.01, 0.01, size=sc.rho.shape))
    sc.bodies[0].twist[2] = -0.02
    return sc


class _OracleRates:
    """J = sum(l . rates) of the oracle with the lists of the base point."""

    def __init__(self, sc):
        self.sc = sc
        self.st = oracle.State(sc)
        self.st.rebuild("brute" if sc.x.shape[0] < 4000 else "cells")

    def J(self, lam, params=None, x=None, u=None, sig=None, rho=None, bodies=None):
        st = self.st
        P = st.params if params is None else params
        x = st.x if x is None else x
        u = st.u if u is None else u
        sig = st.sig if sig is None else sig
        rho = st.rho if rho is None else rho
        b = st.bodies if bodies is None else bodies
        xm, umb, amb = oracle.marker_kinematics(st.mbody, st.mxloc, b, 0.0)
        um, sm = oracle.bce(P, x, u, sig, rho, xm, umb, amb, st.off, st.lst)
        drho, du, ds, macc, _, _ = oracle.rates(P, x, u, sig, rho, xm, um, sm, st.off, st.lst)
        return (np.sum(lam["drho"] * drho) + np.sum(lam["du"] * du) + np.sum(lam["ds"] * ds)
                + np.sum(lam["macc"] * macc))

    def J_abs(self, lam):
        """sum |l . output| at the base point: the FP32 resolution of J is ~1e-7 of it."""
        st = self.st
        xm, umb, amb = oracle.marker_kinematics(st.mbody, st.mxloc, st.bodies, 0.0)
        um, sm = oracle.bce(st.params, st.x, st.u, st.sig, st.rho, xm, umb, amb, st.off, st.lst)
        drho, du, ds, macc, _, _ = oracle.rates(st.params, st.x, st.u, st.sig, st.rho, xm, um, sm,
                                                st.off, st.lst)
        return float(np.sum(np.abs(lam["drho"] * drho)) + np.sum(np.abs(lam["du"] * du))
                     + np.sum(np.abs(lam["ds"] * ds)) + np.sum(np.abs(lam["macc"] * macc)))


def _lam(sc, which, seed):
    rng = np.random.default_rng(seed)
    n, m = sc.x.shape[0], sum(b.markers_local.shape[0] for b in sc.bodies) + sc.fixed.shape[0]
    lam = {"drho": np.zeros(n), "du": np.zeros((n, 3)), "ds": np.zeros((n, 6)), "macc": np.zeros((m, 3))}
    # weights of comparable effect: the stress rates are ~1e6 times the others
    scale = {"drho": 1.0, "du": 1.0, "ds": 1e-4, "macc": 1.0}
    for k in lam:
        if which in (k, "all"):
            lam[k] = rng.normal(size=lam[k].shape) * scale[k]
    return lam


SC_EVAL = _wheel()
INPUTS = ("x", "u", "sig", "rho", "body_c", "body_v", "body_a", "body_theta", "body_w", "E", "nu",
          "rho0", "av_gamma")
BODY_OFF = {"body_c": 0, "body_v": 3, "body_a": 6, "body_theta": 9, "body_w": 12}


def _turned(q, phi):
    """The quaternion q (w, x, y, z) turned by the world-frame rotation vector phi."""
    t = float(np.linalg.norm(phi))
    dq = np.array([1.0, 0.0, 0.0, 0.0]) if t == 0.0 else np.concatenate(
        [[np.cos(t / 2)], np.sin(t / 2) * np.asarray(phi) / t])
    w1, x1, y1, z1 = dq
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


@pytest.fixture(scope="module")
def eval_case():
    sc = SC_EVAL.copy()
    t = crm.from_scene(sc)
    return sc, t, _OracleRates(sc)


def _direction(sc, name, rng):
    """(perturbation kwargs builder, direction, step, adjoint entry)."""
    n = sc.x.shape[0]
    h = sc.params["h"]
    if name in ("x", "u", "sig", "rho"):
        shape = {"x": (n, 3), "u": (n, 3), "sig": (n, 6), "rho": (n,)}[name]
        d = rng.normal(size=shape)
        eps = {"x": 1e-6 * h, "u": 1e-6, "sig": 1e-2, "rho": 1e-3}[name]
        return d, eps
    if name.startswith("body_"):
        return rng.normal(size=3), {"body_c": 1e-6 * h, "body_v": 1e-6, "body_a": 1e-4,
                                    "body_theta": 1e-6, "body_w": 1e-6}[name]
    return np.ones(1), 1e-6 * abs(sc.params[name])


def _perturbed(orc, name, d, e):
    st = orc.st
    if name in ("x", "u", "sig", "rho"):
        return {name: getattr(st, name) + e * d}
    if name.startswith("body_"):
        b = copy.deepcopy(st.bodies)
        if name == "body_c":
            b.pose[0, :3] += e * d
        elif name == "body_v":
            b.twist[0, :3] += e * d
        elif name == "body_a":
            b.acc[0, :3] += e * d
        elif name == "body_theta":
            b.pose[0, 3:] = _turned(b.pose[0, 3:], e * d)
        else:
            b.twist[0, 3:] += e * d
        return {"bodies": b}
    P = dict(st.params)
    P[name] += e * d[0]
    return {"params": P}


def _adjoint_terms(g, name, d):
    if name in ("x", "u", "sig", "rho"):
        key = {"x": "xyz", "u": "vel", "sig": "stress", "rho": "rho"}[name]
        return g[key].reshape(d.shape) * d
    if name.startswith("body_"):
        off = BODY_OFF[name]
        return g["body"][0, off:off + 3] * d
    return np.array([g["param_grads"][name] * d[0]])


@pytest.mark.parametrize("which", ["drho", "du", "ds", "macc"])
def test_rate_vjp_matches_oracle_differences(eval_case, which):
    sc, t, orc = eval_case
    lam = _lam(sc, which, seed=hash(which) % 1000)
    g = t.eval_rates_vjp(lam["drho"], lam["du"], lam["ds"], lam["macc"])
    rng = np.random.default_rng(5)
    j_abs = orc.J_abs(lam)
    bad = []
    for name in INPUTS:
        d, e = _direction(sc, name, rng)
        jp = orc.J(lam, **_perturbed(orc, name, d, e))
        jm = orc.J(lam, **_perturbed(orc, name, d, -e))
        fd = (jp - jm) / (2 * e)
        terms = _adjoint_terms(g, name, d)
        ad, scale = float(terms.sum()), float(np.abs(terms).sum())
        # a parameter derivative can be a small remainder of cancelling terms (the
        # marker accelerations hardly depend on rho0): its floor is the FP32
        # resolution of J per relative change of the parameter
        floor = 1e-6 * j_abs / abs(sc.params[name]) if name in sc.params else 0.0
        if abs(ad - fd) > TOL * scale + floor + 1e-9 * (abs(fd) + 1):
            bad.append((name, ad, fd, scale))
    assert not bad, bad


def test_rate_vjp_of_zero_weights_is_zero(eval_case):
    sc, t, _ = eval_case
    g = t.eval_rates_vjp()
    for k in ("xyz", "vel", "stress", "rho", "body", "params"):
        assert np.all(g[k] == 0.0), k


def test_rate_vjp_rejects_active_domains():
    sc = scenes.wheel_bin(seed=3, nx=20, ny=12, nz=6, wheel_radius=0.05, wheel_width=0.05,
                          n_grousers=6, wheel_x=0.1, active_box=np.array([0.1, 0.1, 0.1]))
    t = crm.from_scene(sc)
    with pytest.raises(crm.CrmError):
        t.eval_rates_vjp(l_drho=np.ones(sc.x.shape[0]))


# ---------------------------------------------------------------------------
# A run of steps: J = sum_s lw_s . wrench_s + lc_s . centre_s
N_RUN, EVERY = 4, 3


def _oracle_run_J(sc, lw, lc, dt, params=None, x=None, u=None, sig=None, rho=None, bodies=None,
                  lfin=None, n_steps=None):
    """J = sum_s lw_s . wrench_s + lc_s . centre_s + lfin . final SPH state (oracle)."""
    s2 = sc.copy()
    if params is not None:
        s2.params = params
    for k, v in (("x", x), ("u", u), ("sig", sig), ("rho", rho)):
        if v is not None:
            setattr(s2, k, v)
    st = oracle.State(s2)
    if bodies is not None:
        st.bodies = bodies
    J = 0.0
    n = lw.shape[0] if n_steps is None else n_steps
    for s in range(n):
        st.step(dt, "brute" if sc.x.shape[0] < 4000 else "cells")
        if lw is not None and len(sc.bodies):
            J += float(np.sum(lw[s, 0] * st.bodies.wrench[0]) + np.sum(lc[s, 0] * st.bodies.pose[0, :3]))
    if lfin is not None:
        J += float(np.sum(lfin["x"] * st.x) + np.sum(lfin["u"] * st.u) + np.sum(lfin["sig"] * st.sig)
                   + np.sum(lfin["rho"] * st.rho))
    return J


def _final_weights(n, seed):
    rng = np.random.default_rng(seed)
    return {"x": rng.normal(size=(n, 3)) * 10.0, "u": rng.normal(size=(n, 3)),
            "sig": rng.normal(size=(n, 6)) * 1e-4, "rho": rng.normal(size=n) * 1e-2}


@pytest.fixture(scope="module")
def run_case():
    sc = _wheel(seed=31, nx=16, ny=12, nz=6)
    sc.params["mu_2"] = sc.params["mu_s"]
    sc.params["skin"] = 0.0            # differentiable runs search the cells every step
    t = crm.from_scene(sc)
    dt = sc.dt
    w, q = t.adjoint_forward(dt, N_RUN, EVERY)
    rng = np.random.default_rng(7)
    lw = rng.normal(size=(N_RUN, 1, 6))
    lw[:, :, 3:] *= 10.0
    lc = rng.normal(size=(N_RUN, 1, 3)) * 1e3
    lf = _final_weights(sc.x.shape[0], 8)
    g = t.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    return sc, t, dt, w, q, lw, lc, g, lf


def test_run_forward_matches_plain_steps(run_case):
    sc, t, dt, w, q, *_ = run_case
    t2 = crm.from_scene(sc.copy())
    for s in range(N_RUN):
        t2.step(dt, 1)
        f, tq = t2.body_wrench(0)
        np.testing.assert_array_equal(w[s, 0], np.concatenate([f, tq]))
        pose, _ = t2.body_state(0)
        np.testing.assert_array_equal(q[s, 0], pose)


@pytest.mark.parametrize("name", ["E", "nu", "rho0", "mu_s", "cohesion", "av_gamma", "x", "u",
                                  "sig", "rho", "body_c", "body_v", "body_theta", "body_w"])
def test_run_gradient_matches_oracle_differences(run_case, name):
    sc, t, dt, w, q, lw, lc, g, lf = run_case
    rng = np.random.default_rng(11)
    base = oracle.State(sc)
    n = sc.x.shape[0]
    h = sc.params["h"]
    if name in ("x", "u", "sig", "rho"):
        shape = {"x": (n, 3), "u": (n, 3), "sig": (n, 6), "rho": (n,)}[name]
        d = rng.normal(size=shape)
        e = {"x": 1e-6 * h, "u": 1e-6, "sig": 1e-2, "rho": 1e-3}[name]
        arr = getattr(base, name)
        jp = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr + e * d})
        jm = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr - e * d})
        key = {"x": "xyz", "u": "vel", "sig": "stress", "rho": "rho"}[name]
        terms = g[key].reshape(d.shape) * d
    elif name.startswith("body_"):
        d = rng.normal(size=3)
        e = 1e-6 * h if name == "body_c" else 1e-6
        bp, bm = copy.deepcopy(base.bodies), copy.deepcopy(base.bodies)
        if name == "body_c":
            bp.pose[0, :3] += e * d
            bm.pose[0, :3] -= e * d
        elif name == "body_v":
            bp.twist[0, :3] += e * d
            bm.twist[0, :3] -= e * d
        elif name == "body_theta":
            bp.pose[0, 3:] = _turned(bp.pose[0, 3:], e * d)
            bm.pose[0, 3:] = _turned(bm.pose[0, 3:], -e * d)
        else:
            bp.twist[0, 3:] += e * d
            bm.twist[0, 3:] -= e * d
        jp = _oracle_run_J(sc, lw, lc, dt, bodies=bp, lfin=lf)
        jm = _oracle_run_J(sc, lw, lc, dt, bodies=bm, lfin=lf)
        off = BODY_OFF[name]
        terms = g["body"][0, off:off + 3] * d
    else:
        e = 1e-6 * abs(sc.params[name])
        pp, pm = dict(sc.params), dict(sc.params)
        pp[name] += e
        pm[name] -= e
        if name == "mu_s":   # a constant friction coefficient: mu_2 follows mu_s
            pp["mu_2"], pm["mu_2"] = pp["mu_s"], pm["mu_s"]
        jp = _oracle_run_J(sc, lw, lc, dt, params=pp, lfin=lf)
        jm = _oracle_run_J(sc, lw, lc, dt, params=pm, lfin=lf)
        terms = np.array([g["param_grads"][name]])
    fd = (jp - jm) / (2 * e)
    ad, scale = float(terms.sum()), float(np.abs(terms).sum())
    assert abs(ad - fd) <= RUN_TOL * max(scale, abs(fd)) + 1e-9, (name, ad, fd, scale)


def test_run_backward_restores_the_final_state(run_case):
    sc, t, dt, w, q, *_ = run_case
    pose, _ = t.body_state(0)
    np.testing.assert_array_equal(pose, q[-1, 0])


def test_run_rejects_unsupported_configurations():
    sc = _wheel(seed=41, nx=16, ny=12, nz=6)
    sc.params["skin"] = 0.0
    sc.boxes.append(scenes.ActiveBox(0, np.array([0.1, 0.1, 0.1]), np.zeros(3)))
    with pytest.raises(crm.CrmError):                # active domains
        crm.from_scene(sc).adjoint_forward(sc.dt, 2, 1)
    sc.boxes.clear()
    sc.params["skin"] = 0.1                          # a Verlet skin
    with pytest.raises(crm.CrmError):
        crm.from_scene(sc).adjoint_forward(sc.dt, 2, 1)
    t2 = crm.from_scene(_wheel(seed=42, nx=16, ny=12, nz=6))
    with pytest.raises(crm.CrmError):                # nothing recorded
        t2.adjoint_backward(None, None)


def test_autograd_function_matches_the_c_abi(run_case):
    import torch

    from paper_2507_05643_b300.autograd import TerrainRun, scene_params
    sc, t, dt, w, q, lw, lc, g, lf = run_case
    params = scene_params(sc).requires_grad_(True)
    state = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
             for a in (sc.x, sc.u, sc.sig, sc.rho)]
    W, Cc, xT, uT, sT, rT = TerrainRun.apply(params, *state, sc, N_RUN, EVERY)
    np.testing.assert_array_equal(W.detach().numpy(), w)
    J = ((W * torch.from_numpy(lw)).sum() + (Cc * torch.from_numpy(lc)).sum()
         + (xT * torch.from_numpy(lf["x"])).sum() + (uT * torch.from_numpy(lf["u"])).sum()
         + (sT * torch.from_numpy(lf["sig"])).sum() + (rT * torch.from_numpy(lf["rho"])).sum())
    J.backward()
    # the same sweep; FP64 atomics order the parameter and body sums freely
    np.testing.assert_allclose(params.grad.numpy(), g["params"], rtol=1e-6)
    for a, key in zip(state, ("xyz", "vel", "stress", "rho")):
        np.testing.assert_allclose(a.grad.numpy(), g[key], rtol=1e-4,
                                   atol=1e-6 * np.abs(g[key]).max())


# ---------------------------------------------------------------------------
# Variants of the rate evaluation: Wendland kernel, bilateral and no viscosity


@pytest.mark.parametrize("variant", ["wendland", "bilateral", "no_av"])
def test_rate_vjp_variants_match_oracle_differences(variant):
    sc = _wheel(seed=51, nx=20, ny=14, nz=7)
    if variant == "wendland":
        sc.params["kernel"] = 1
    elif variant == "bilateral":
        sc.params["av_mode"] = 1
    else:
        sc.params["av_mode"] = 0
    t = crm.from_scene(sc)
    orc = _OracleRates(sc)
    lam = _lam(sc, "all", seed=3)
    g = t.eval_rates_vjp(lam["drho"], lam["du"], lam["ds"], lam["macc"])
    rng = np.random.default_rng(9)
    j_abs = orc.J_abs(lam)
    bad = []
    for name in INPUTS:
        d, e = _direction(sc, name, rng)
        fd = (orc.J(lam, **_perturbed(orc, name, d, e)) - orc.J(lam, **_perturbed(orc, name, d, -e))) / (2 * e)
        terms = _adjoint_terms(g, name, d)
        ad, scale = float(terms.sum()), float(np.abs(terms).sum())
        floor = 1e-6 * j_abs / abs(sc.params[name]) if name in sc.params else 0.0
        if abs(ad - fd) > TOL * scale + floor + 1e-9 * (abs(fd) + 1):
            bad.append((name, ad, fd, scale))
    assert not bad, bad


def test_run_without_bodies_matches_oracle_differences():
    """A walled block without bodies, J on the final SPH state only."""
    sc = scenes.settling_block(seed=61, n=8, box=0.14)
    rng = np.random.default_rng(61)
    sc.u = rng.uniform(-0.05, 0.05, size=sc.u.shape)
    sc.sig = np.zeros_like(sc.sig)
    sc.sig[:, :3] = -rng.uniform(500.0, 2000.0, size=(sc.x.shape[0], 3))
    sc.sig[:, 3:] = rng.uniform(-100.0, 100.0, size=(sc.x.shape[0], 3))
    sc.params["skin"] = 0.0
    sc.params["cohesion"] = 200.0
    n_steps = 3
    t = crm.from_scene(sc)
    t.adjoint_forward(sc.dt, n_steps, 2)
    lf = _final_weights(sc.x.shape[0], 62)
    g = t.adjoint_backward(None, None, lf["x"], lf["u"], lf["sig"], lf["rho"])
    assert g["body"].shape == (0, 18)
    h = sc.params["h"]
    bad = []
    for name in ("x", "u", "sig", "rho", "E", "rho0", "mu_s", "cohesion"):
        if name in ("x", "u", "sig", "rho"):
            shape = {"x": (-1, 3), "u": (-1, 3), "sig": (-1, 6), "rho": (-1,)}[name]
            arr = getattr(sc, name)
            d = rng.normal(size=arr.shape)
            e = {"x": 1e-6 * h, "u": 1e-6, "sig": 1e-2, "rho": 1e-3}[name]
            jp = _oracle_run_J(sc, None, None, sc.dt, lfin=lf, n_steps=n_steps, **{name: arr + e * d})
            jm = _oracle_run_J(sc, None, None, sc.dt, lfin=lf, n_steps=n_steps, **{name: arr - e * d})
            key = {"x": "xyz", "u": "vel", "sig": "stress", "rho": "rho"}[name]
            terms = g[key].reshape(d.shape) * d
        else:
            e = 1e-6 * abs(sc.params[name])
            pp, pm = dict(sc.params), dict(sc.params)
            pp[name] += e
            pm[name] -= e
            if name == "mu_s":
                pp["mu_2"], pm["mu_2"] = pp["mu_s"], pm["mu_s"]
            jp = _oracle_run_J(sc, None, None, sc.dt, params=pp, lfin=lf, n_steps=n_steps)
            jm = _oracle_run_J(sc, None, None, sc.dt, params=pm, lfin=lf, n_steps=n_steps)
            terms = np.array([g["param_grads"][name]])
        fd = (jp - jm) / (2 * e)
        ad, scale = float(terms.sum()), float(np.abs(terms).sum())
        if abs(ad - fd) > RUN_TOL * max(scale, abs(fd)) + 1e-9:
            bad.append((name, ad, fd, scale))
    assert not bad, bad


def test_resident_tape_matches_the_checkpointed_run(run_case):
    """every = 0 keeps every step's tape (no checkpoints, no re-run): the same
    recorded run and the same sweep, so the same gradients."""
    sc, t, dt, w, q, lw, lc, g, lf = run_case
    t2 = crm.from_scene(sc)
    w2, q2 = t2.adjoint_forward(dt, N_RUN, 0)
    np.testing.assert_array_equal(w2, w)
    np.testing.assert_array_equal(q2, q)
    g2 = t2.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    np.testing.assert_allclose(g2["params"], g["params"], rtol=1e-9)
    for key in ("xyz", "vel", "stress", "rho"):
        np.testing.assert_allclose(g2[key], g[key], rtol=1e-5, atol=1e-7 * np.abs(g[key]).max())


@pytest.mark.parametrize("name", ["mu_s", "mu_2", "I0", "grain_d", "E", "rho0", "sig", "x"])
def test_run_gradient_with_mu_i_matches_oracle_differences(name):
    """The rate-dependent friction mu(I) (mu_2 != mu_s): its constants, and the
    stress at t_n through the shear rate."""
    sc = _wheel(seed=71, nx=16, ny=12, nz=6)
    sc.params["skin"] = 0.0
    sc.params["mu_2"] = sc.params["mu_s"] + 0.3
    sc.bodies[0].pose[2] -= 0.004                    # deeper: more of the soil yields
    t = crm.from_scene(sc)
    dt = sc.dt
    t.adjoint_forward(dt, N_RUN, EVERY)
    rng = np.random.default_rng(13)
    lw = rng.normal(size=(N_RUN, 1, 6))
    lc = rng.normal(size=(N_RUN, 1, 3)) * 1e3
    lf = _final_weights(sc.x.shape[0], 14)
    g = t.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    if name in ("sig", "x"):
        arr = getattr(sc, name)
        d = rng.normal(size=arr.shape)
        e = 1e-2 if name == "sig" else 1e-6 * sc.params["h"]
        jp = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr + e * d})
        jm = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr - e * d})
        terms = g["stress" if name == "sig" else "xyz"].reshape(d.shape) * d
    else:
        e = 1e-6 * abs(sc.params[name])
        pp, pm = dict(sc.params), dict(sc.params)
        pp[name] += e
        pm[name] -= e
        jp = _oracle_run_J(sc, lw, lc, dt, params=pp, lfin=lf)
        jm = _oracle_run_J(sc, lw, lc, dt, params=pm, lfin=lf)
        terms = np.array([g["param_grads"][name]])
    fd = (jp - jm) / (2 * e)
    ad, scale = float(terms.sum()), float(np.abs(terms).sum())
    if name in ("mu_2", "I0", "grain_d"):     # the rate branch is exercised
        assert abs(fd) * abs(sc.params[name]) > 1e-6 * abs(jp), (name, fd, jp)
    assert abs(ad - fd) <= RUN_TOL * max(scale, abs(fd)) + 1e-9, (name, ad, fd, scale)


# ---------------------------------------------------------------------------
# A body with all six DOFs free (Euler's equations with unequal moments)


@pytest.fixture(scope="module")
def six_dof_case():
    sc = scenes.sphere_drop(seed=81, nx=16, ny=16, nz=8, radius=0.04)
    sc.params["skin"] = 0.0
    b = sc.bodies[0]
    b.inertia = b.inertia * np.array([1.0, 2.0, 4.0])   # unequal moments: w x I w != 0
    b.twist[3:] = [40.0, -30.0, 25.0]                    # fast: the gyroscopic terms count
    b.pose[2] -= 0.006                                   # in contact with the bed
    t = crm.from_scene(sc)
    t.adjoint_forward(sc.dt, N_RUN, EVERY)
    rng = np.random.default_rng(17)
    lw = rng.normal(size=(N_RUN, 1, 6))
    lw[:, :, 3:] *= 10.0
    lc = rng.normal(size=(N_RUN, 1, 3)) * 1e3
    lf = _final_weights(sc.x.shape[0], 18)
    g = t.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    return sc, g, lw, lc, lf


@pytest.mark.parametrize("name", ["E", "mu_s", "x", "sig", "body_c", "body_v", "body_theta",
                                  "body_w", "body_a", "body_alpha"])
def test_run_six_dof_gradient_matches_oracle_differences(six_dof_case, name):
    sc, g, lw, lc, lf = six_dof_case
    dt = sc.dt
    rng = np.random.default_rng(19)
    base = oracle.State(sc)
    if name in ("x", "sig"):
        arr = getattr(sc, name)
        d = rng.normal(size=arr.shape)
        e = 1e-2 if name == "sig" else 1e-6 * sc.params["h"]
        jp = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr + e * d})
        jm = _oracle_run_J(sc, lw, lc, dt, lfin=lf, **{name: arr - e * d})
        terms = g["stress" if name == "sig" else "xyz"].reshape(d.shape) * d
    elif name.startswith("body_"):
        d = rng.normal(size=3)
        e = 1e-6 * sc.params["h"] if name == "body_c" else 1e-6
        bp, bm = copy.deepcopy(base.bodies), copy.deepcopy(base.bodies)
        for bb, sgn in ((bp, 1.0), (bm, -1.0)):
            if name == "body_c":
                bb.pose[0, :3] += sgn * e * d
            elif name == "body_v":
                bb.twist[0, :3] += sgn * e * d
            elif name == "body_theta":
                bb.pose[0, 3:] = _turned(bb.pose[0, 3:], sgn * e * d)
            elif name == "body_w":
                bb.twist[0, 3:] += sgn * e * d
            elif name == "body_a":
                bb.acc[0, :3] += sgn * e * d
            else:
                bb.acc[0, 3:] += sgn * e * d
        jp = _oracle_run_J(sc, lw, lc, dt, bodies=bp, lfin=lf)
        jm = _oracle_run_J(sc, lw, lc, dt, bodies=bm, lfin=lf)
        off = dict(BODY_OFF, body_alpha=15)[name]
        terms = g["body"][0, off:off + 3] * d
    else:
        e = 1e-6 * abs(sc.params[name])
        pp, pm = dict(sc.params), dict(sc.params)
        pp[name] += e
        pm[name] -= e
        if name == "mu_s":
            pp["mu_2"], pm["mu_2"] = pp["mu_s"], pm["mu_s"]
        jp = _oracle_run_J(sc, lw, lc, dt, params=pp, lfin=lf)
        jm = _oracle_run_J(sc, lw, lc, dt, params=pm, lfin=lf)
        terms = np.array([g["param_grads"][name]])
    fd = (jp - jm) / (2 * e)
    ad, scale = float(terms.sum()), float(np.abs(terms).sum())
    assert abs(ad - fd) <= RUN_TOL * max(scale, abs(fd)) + 1e-9, (name, ad, fd, scale)


# ---------------------------------------------------------------------------
# Against the oracle's own FP64 adjoint (oracle/adjoint.py, pinned to the C
# oracle by tests/test_oracle_adjoint.py): every entry of every gradient, not
# one direction.  Bars: the relative L2 error of each array, the largest entry
# error against the array's largest entry, each parameter gradient against its
# own size (FP32 sweep of an FP32 trajectory against FP64 throughout).
# (measured on a B300: 1e-7 to 9e-7 everywhere but the six-DOF orientation, 7.5e-6)
ORACLE_REL = 5e-5        # relative L2 error of an array / error of a parameter gradient
ORACLE_MAX = 5e-5        # largest entry error / largest entry


def _against_oracle_adjoint(sc, g, lw, lc, lf, n_steps, params):
    from oracle import adjoint as oadj
    _, _, o = oadj.run_gradients(sc, sc.dt, n_steps, lw, lc, lf, mode="brute")
    errs, bad = {}, []
    pairs = [("xyz", "x"), ("vel", "u"), ("stress", "sig"), ("rho", "rho")]
    arrays = {k: (np.asarray(g[k], float).reshape(o[ko].shape), o[ko]) for k, ko in pairs}
    if len(sc.bodies):
        b = np.asarray(g["body"], float)[0]
        arrays.update({"body_c": (b[0:3], o["body_c"][0]), "body_v": (b[3:6], o["body_v"][0]),
                       "body_a": (b[6:9], o["body_acc"][0, :3]),
                       "body_theta": (b[9:12], o["body_theta"][0]),
                       "body_w": (b[12:15], o["body_w"][0]),
                       "body_alpha": (b[15:18], o["body_acc"][0, 3:])})
    for k, (a, r) in arrays.items():
        nr = float(np.linalg.norm(r))
        if nr == 0.0:
            continue
        rel = float(np.linalg.norm(a - r)) / nr
        mx = float(np.abs(a - r).max()) / float(np.abs(r).max())
        errs[k] = (rel, mx)
        if rel > ORACLE_REL or mx > ORACLE_MAX:
            bad.append(k)
    for k in params:
        a, r = float(g["param_grads"][k]), float(o["params"][k])
        rel = abs(a - r) / max(abs(r), 1e-300)
        errs[k] = rel
        if rel > ORACLE_REL:
            bad.append(k)
    print("errors against the oracle adjoint:", errs)
    assert not bad, (bad, errs)


def test_run_gradients_match_the_oracle_adjoint(run_case):
    sc, t, dt, w, q, lw, lc, g, lf = run_case
    _against_oracle_adjoint(sc, g, lw, lc, lf, N_RUN, ("E", "nu", "rho0", "mu_s", "cohesion",
                                                      "av_gamma"))


def test_six_dof_gradients_match_the_oracle_adjoint(six_dof_case):
    sc, g, lw, lc, lf = six_dof_case
    _against_oracle_adjoint(sc, g, lw, lc, lf, N_RUN, ("E", "nu", "rho0", "mu_s", "av_gamma"))


def test_mu_i_gradients_match_the_oracle_adjoint():
    sc = _wheel(seed=71, nx=16, ny=12, nz=6)
    sc.params["skin"] = 0.0
    sc.params["mu_2"] = sc.params["mu_s"] + 0.3
    sc.bodies[0].pose[2] -= 0.004
    t = crm.from_scene(sc)
    t.adjoint_forward(sc.dt, N_RUN, EVERY)
    rng = np.random.default_rng(13)
    lw = rng.normal(size=(N_RUN, 1, 6))
    lc = rng.normal(size=(N_RUN, 1, 3)) * 1e3
    lf = _final_weights(sc.x.shape[0], 14)
    g = t.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    _against_oracle_adjoint(sc, g, lw, lc, lf, N_RUN, ("E", "mu_s", "mu_2", "I0", "grain_d",
                                                      "cohesion"))

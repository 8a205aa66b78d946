"""Pins of the oracle's own FP64 adjoint (``oracle/adjoint.py``, a PyTorch CPU
restatement of the oracle step differentiated by autograd) to the C oracle:

* its forward steps reproduce ``orc_step`` to FP64 rounding (state, body pose
  and twist, wrench) on scenes that take every branch: walls and a driven
  wheel, the rate-dependent friction mu(I) with yielding, the Wendland kernel
  with bilateral viscosity, a body with all six DOFs free;
* its gradients of J = sum lw . wrench + lc . centre + lfin . final state match
  FP64 central differences of the C oracle's runs for every input group.

The C oracle is pinned by ``test_oracle_pins.py``; agreement with it in value
and in finite differences is what makes this adjoint a reference for the CUDA
reverse sweep.
"""
import copy

import numpy as np
import pytest

import oracle
import scenes
from oracle import adjoint as oadj

N_STEPS = 3


def _wheel(seed=21, nx=12, ny=10, nz=6, mu_i=False):
    sc = scenes.wheel_bin(seed=seed, nx=nx, ny=ny, nz=nz, wheel_radius=0.05, wheel_width=0.05,
                          n_grousers=8, wheel_x=0.06)
    sc.bodies[0].pose[2] -= 0.006
    rng = np.random.default_rng(seed)
    sc.u = rng.uniform(-0.05, 0.05, size=sc.u.shape)
    sc.sig = sc.sig + rng.uniform(-300.0, 300.0, size=sc.sig.shape)
    sc.rho = sc.params["rho0"] * (1 + rng.uniform(-0.01, 0.01, size=sc.rho.shape))
    sc.bodies[0].twist[2] = -0.02
    if mu_i:
        sc.params["mu_2"] = sc.params["mu_s"] + 0.3
        sc.params["cohesion"] = 0.0
    return sc


def _sphere(seed=81):
    sc = scenes.sphere_drop(seed=seed, nx=10, ny=10, nz=6, radius=0.03)
    b = sc.bodies[0]
    b.inertia = b.inertia * np.array([1.0, 2.0, 4.0])
    b.twist[3:] = [40.0, -30.0, 25.0]
    b.pose[2] -= 0.006
    return sc


def _scene(name):
    if name == "wheel":
        return _wheel()
    if name == "mu_i":
        return _wheel(seed=23, mu_i=True)
    if name == "wendland":
        sc = _wheel(seed=25)
        sc.params["kernel"] = 1
        sc.params["av_mode"] = 1
        return sc
    return _sphere()


SCENES = ["wheel", "mu_i", "wendland", "six_dof"]


def _c_run(sc, n, params=None, x=None, u=None, sig=None, rho=None, bodies=None):
    s2 = sc.copy()
    if params is not None:
        s2.params = params
    for k, v in (("x", x), ("u", u), ("sig", sig), ("rho", rho)):
        if v is not None:
            setattr(s2, k, v)
    st = oracle.State(s2)
    if bodies is not None:
        st.bodies = bodies
    W, Q = [], []
    for _ in range(n):
        st.step(sc.dt, "brute")
        W.append(st.bodies.wrench[:st.bodies.n].copy())
        Q.append(st.bodies.pose[:st.bodies.n].copy())
    return st, np.array(W), np.array(Q)


@pytest.mark.parametrize("name", SCENES)
def test_forward_reproduces_the_c_oracle(name):
    sc = _scene(name)
    st, W, Q = _c_run(sc, N_STEPS)
    r = oadj.Run(sc, "brute")
    w, q = r.forward(sc.dt, N_STEPS)
    x, u, s, rho, B = r.final
    sig_scale = np.abs(st.sig).max()
    np.testing.assert_allclose(x.numpy(), st.x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u.numpy(), st.u, rtol=0, atol=1e-12 * max(np.abs(st.u).max(), 1))
    np.testing.assert_allclose(s.numpy(), st.sig, rtol=0, atol=1e-11 * sig_scale)
    np.testing.assert_allclose(rho.numpy(), st.rho, rtol=1e-13)
    np.testing.assert_allclose(q, Q, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, W, rtol=0, atol=1e-10 * max(np.abs(W).max(), 1e-3))
    np.testing.assert_allclose(B.twist.numpy(), st.bodies.twist[:1], rtol=0, atol=1e-12)
    if name == "mu_i":   # the rate branch and the cone are both taken
        sn = sc.sig
        tb = lambda a: np.sqrt(0.5 * (np.sum((a[:, :3] + (-a[:, :3].sum(1) / 3)[:, None]) ** 2, 1)
                                      + 2 * np.sum(a[:, 3:] ** 2, 1)))
        assert np.sum(tb(st.sig) < tb(sn) * 0.999) > 0


def _turned(q, phi):
    t = float(np.linalg.norm(phi))
    dq = np.concatenate([[np.cos(t / 2)], np.sin(t / 2) * np.asarray(phi) / t])
    w1, x1, y1, z1 = dq
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _weights(sc, seed):
    rng = np.random.default_rng(seed)
    n = sc.x.shape[0]
    lw = rng.normal(size=(N_STEPS, 1, 6))
    lw[:, :, 3:] *= 10.0
    lc = rng.normal(size=(N_STEPS, 1, 3)) * 1e3
    lf = {"x": rng.normal(size=(n, 3)) * 10.0, "u": rng.normal(size=(n, 3)),
          "sig": rng.normal(size=(n, 6)) * 1e-4, "rho": rng.normal(size=n) * 1e-2}
    return lw, lc, lf


def _J(sc, lw, lc, lf, **kw):
    st, W, Q = _c_run(sc, N_STEPS, **kw)
    J = float(np.sum(lw * W) + np.sum(lc * Q[:, :, :3]))
    return J + float(np.sum(lf["x"] * st.x) + np.sum(lf["u"] * st.u) + np.sum(lf["sig"] * st.sig)
                     + np.sum(lf["rho"] * st.rho))


_GRADS = {}


def _grads(name):
    if name not in _GRADS:
        sc = _scene(name)
        lw, lc, lf = _weights(sc, 5)
        _, _, g = oadj.run_gradients(sc, sc.dt, N_STEPS, lw, lc, lf, mode="brute")
        _GRADS[name] = (sc, lw, lc, lf, g)
    return _GRADS[name]


CASES = ([("wheel", k) for k in ("E", "nu", "rho0", "mu_s", "cohesion", "av_gamma", "x", "u",
                                 "sig", "rho", "body_c", "body_v", "body_theta", "body_w")]
         + [("mu_i", k) for k in ("mu_s", "mu_2", "I0", "grain_d", "sig")]
         + [("wendland", k) for k in ("E", "x", "u")]
         + [("six_dof", k) for k in ("E", "x", "body_c", "body_v", "body_theta", "body_w",
                                     "body_acc")])


@pytest.mark.parametrize("scene,name", CASES)
def test_gradient_matches_c_oracle_differences(scene, name):
    sc, lw, lc, lf, g = _grads(scene)
    rng = np.random.default_rng(sum(map(ord, scene + name)))
    base = oracle.State(sc)
    h = sc.params["h"]
    if name in ("x", "u", "sig", "rho"):
        arr = getattr(base, name)
        d = rng.normal(size=arr.shape)
        e = {"x": 1e-6 * h, "u": 1e-6, "sig": 1e-2, "rho": 1e-3}[name]
        jp = _J(sc, lw, lc, lf, **{name: arr + e * d})
        jm = _J(sc, lw, lc, lf, **{name: arr - e * d})
        terms = g[name].reshape(d.shape) * d
    elif name.startswith("body_"):
        d = rng.normal(size=6 if name == "body_acc" else 3)
        # J depends weakly on the marker accelerations' start values: a larger
        # step keeps the differences' rounding below the bar
        e = 1e-6 * h if name == "body_c" else (1e-4 if name == "body_acc" else 1e-6)
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
            else:
                bb.acc[0] += sgn * e * d
        jp = _J(sc, lw, lc, lf, bodies=bp)
        jm = _J(sc, lw, lc, lf, bodies=bm)
        terms = g[name][0] * d
    else:
        # the viscosity constant enters J weakly (rounding of the differences
        # dominates at a 1e-6 step; the 1e-4 difference agrees to 3e-8)
        e = (1e-4 if name == "av_gamma" else 1e-6) * abs(sc.params[name])
        pp, pm = dict(sc.params), dict(sc.params)
        pp[name] += e
        pm[name] -= e
        if name == "mu_s" and sc.params["mu_2"] == sc.params["mu_s"]:
            pp["mu_2"], pm["mu_2"] = pp["mu_s"], pm["mu_s"]   # constant friction
        jp = _J(sc, lw, lc, lf, params=pp)
        jm = _J(sc, lw, lc, lf, params=pm)
        terms = np.array([g["params"][name]])
    fd = (jp - jm) / (2 * e)
    ad, scale = float(terms.sum()), float(np.abs(terms).sum())
    if scene == "mu_i" and name in ("mu_2", "I0", "grain_d"):   # the rate branch matters
        assert abs(fd) * abs(sc.params[name]) > 1e-6 * abs(jp), (name, fd, jp)
    assert abs(ad - fd) <= 1e-6 * max(scale, abs(fd)) + 1e-12, (scene, name, ad, fd, scale)


def test_forward_pin_catches_a_planted_slip(monkeypatch):
    """A slip of 1e-4 in the stress rate moves the restated step off the C
    oracle by far more than the forward pin's tolerance."""
    sc = _scene("wheel")
    st, _, _ = _c_run(sc, 1)
    orig = oadj._rates

    def bad(*a, **k):
        drho, du, ds, macc = orig(*a, **k)
        return drho, du, ds * 1.0001, macc
    monkeypatch.setattr(oadj, "_rates", bad)
    r = oadj.Run(sc, "brute")
    r.forward(sc.dt, 1)
    assert np.abs(r.final[2].numpy() - st.sig).max() > 1e-9 * np.abs(st.sig).max()

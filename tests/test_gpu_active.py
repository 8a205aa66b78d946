"""Active domains (Sec. 3.2, Alg. 3) on the GPU against the FP64 oracle.

Flags and counts are integer work: the Active / Extended-Active counts equal the
oracle's except for particles whose FP64 box-frame coordinate lies within 1e-7 m
of a face (the GPU holds positions as FP32 cell offsets, so a particle that close
may fall on either side).  States: particles never active stay bit-for-bit at
their FP32 inputs; the rest are compared with the short-horizon bars of the
plain path.
"""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu
crm = pytest.importorskip("paper_2507_05643_b300")


def _scene(seed=51, carrier_v=(20.0, 0.0, 0.0), carrier_z=None, t_delay=-1.0, half=(0.06, 0.06, 0.06)):
    sc = scenes.wheel_bin(seed=seed, nx=60, ny=24, nz=10, wheel_radius=0.06, wheel_width=0.06,
                          n_grousers=6, wheel_x=0.42, dt=1e-4)
    sc.bodies[0].pose[2] -= 0.004
    z = 0.05 if carrier_z is None else carrier_z
    carrier = scenes.Body(np.zeros((0, 3)), np.array([0.08, 0.12, z, 1, 0, 0, 0.0]),
                          np.array([*carrier_v, 0, 0, 0.0]), 1.0, 0)
    sc.bodies.append(carrier)
    sc.boxes = [scenes.ActiveBox(0, np.array([0.09, 0.06, 0.09]), np.zeros(3)),
                scenes.ActiveBox(1, np.array(half), np.zeros(3))]
    sc.t_delay = t_delay
    return sc


def _near_face(x, boxes, pose, h, tol=1e-7):
    """Particles within tol of a face of a box or of its 2h-grown box."""
    near = np.zeros(x.shape[0], bool)
    for b in boxes:
        p = pose[b.body]
        w, qx, qy, qz = p[3:]
        R = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - w * qz), 2 * (qx * qz + w * qy)],
                      [2 * (qx * qy + w * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - w * qx)],
                      [2 * (qx * qz - w * qy), 2 * (qy * qz + w * qx), 1 - 2 * (qx * qx + qy * qy)]])
        l = (x - (p[:3] + R @ b.offset)) @ R
        for e in (b.half_extents, b.half_extents + 2 * h):
            near |= np.any(np.abs(np.abs(l) - e) < tol, axis=1)
    return near


@pytest.mark.parametrize("t_delay", [-1.0, 0.00045])
def test_active_domain_steps_match_oracle(t_delay):
    sc = _scene(t_delay=t_delay)
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    t.step(sc.dt, 0)                  # commit: the state is now held as FP32 cell offsets
    x0, u0, s0, r0 = t.particles()
    n = 60
    t.step(sc.dt, n)
    st.run(n)
    na, ne, nb = t.counts()
    fl = st.flags
    assert fl is not None
    near = _near_face(st.x, sc.boxes, st.bodies.pose, sc.params["h"])
    oa, oe = int((fl == 2).sum()), int((fl == 1).sum())
    assert abs(na - oa) <= near.sum() and abs(ne - oe) <= near.sum(), (na, oa, ne, oe, near.sum())
    assert na > 500 and ne > 200
    xyz, vel, sig, rho = t.particles()
    d0 = sc.params["d0"]
    dx = np.max(np.abs(xyz - st.x)) / d0
    ds = np.sqrt(np.mean((sig - st.sig) ** 2)) / (sc.params["rho0"] * 9.81 * 0.1)
    print("active: counts", (na, ne, nb), "oracle", (oa, oe), "dx/d0", dx, "dsig", ds)
    assert dx < 1e-4 and ds < 1e-4
    if t_delay < 0:
        # particles the boxes never reached are exactly their FP32 inputs
        moved = np.any(np.abs(st.x - sc.x) > 0, axis=1) | np.any(np.abs(st.sig - sc.sig) > 0, axis=1)
        frozen = ~moved
        assert frozen.sum() > 1000
        assert np.array_equal(xyz[frozen], x0[frozen]) and np.array_equal(sig[frozen], s0[frozen])
    F, _ = t.body_wrench(0)
    Fo = st.bodies.wrench[0, :3]
    assert np.linalg.norm(F - Fo) <= 1e-3 * np.linalg.norm(Fo) + 1e-9


def test_active_capacity_shrinks_then_grows():
    """A box that starts in the air (few particles) and then descends into the soil:
    the working arrays shrink at an S_I boundary and must grow again when the box
    fills -- the step that overflows is abandoned and redone, so the result still
    matches the oracle, which has no capacities."""
    sc = _scene(seed=52, carrier_v=(0.0, 0.0, -20.0), carrier_z=0.25, half=(0.08, 0.08, 0.05))
    sc.params["shrink_interval"] = 5
    p = crm.params_from_dict(sc.params, sc.domain_min, sc.domain_max)
    p.shrink_interval = 5
    t = crm.Terrain(p)
    t.add_sph(sc.x, sc.u, sc.sig, sc.rho)
    t.add_fixed_bce(sc.fixed)
    for b in sc.bodies:
        t.add_rigid_body(b.markers_local, b.pose, b.twist, b.mass, b.dof_mask)
    for bx in sc.boxes:
        t.add_active_box(bx.body, bx.half_extents, bx.offset, sc.t_delay)
    st = oracle.State(sc)
    seen = []
    for k in range(16):
        t.step(sc.dt, 5)
        st.run(5)
        seen.append(t.counts()[0])
    assert seen[-1] > 2 * max(seen[0], 1), seen
    xyz, vel, sig, rho = t.particles()
    assert np.max(np.abs(xyz - st.x)) / sc.params["d0"] < 1e-4
    na = t.counts()[0]
    assert abs(na - int((st.flags == 2).sum())) <= _near_face(st.x, sc.boxes, st.bodies.pose,
                                                               sc.params["h"]).sum()


def test_active_eval_rates_match_oracle():
    sc = _scene(seed=53)
    rng = np.random.default_rng(53)
    sc.u = rng.uniform(-0.05, 0.05, size=sc.u.shape)
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    drho, du, ds, macc, mvel, msig = t.eval_rates()
    o_drho, o_du, o_ds, o_macc, scale, _, _ = st.eval_rates(want_scale=True)
    got = np.concatenate([drho[:, None], du, ds], axis=1).astype(np.float64)
    ref = np.concatenate([o_drho[:, None], o_du, o_ds], axis=1)
    act = st.integrate.astype(bool)
    near = _near_face(st.x, sc.boxes, st.bodies.pose, sc.params["h"], tol=1e-6)
    ok = ~near
    assert np.all(np.abs(got - ref)[act & ok] <= 1e-5 * scale[act & ok] + 1e-30)
    assert np.all(got[~act & ok] == 0)


def test_strip_window_far_from_origin_matches_oracle():
    """The large-scale active-domain case (10 km strip at 0.025 m, four-wheel
    kinematic rover at 1 m/s, a 1 m active box per wheel) on a 20 m window
    around the rover at x = 5000 m: active / extended counts, particle states and
    wheel wrenches follow the oracle; terrain outside the boxes stays frozen."""
    sc = scenes.strip(x_window=(4995.0, 5015.0))
    sc.t_delay = -1.0          # boxes in force from the first step
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    t.step(sc.dt, 0)
    x0, _, s0, _ = t.particles()
    n = 20
    t.step(sc.dt, n)
    st.run(n)
    na, ne, nb = t.counts()
    near = _near_face(st.x, sc.boxes, st.bodies.pose, sc.params["h"])
    oa, oe = int((st.flags == 2).sum()), int((st.flags == 1).sum())
    assert abs(na - oa) <= near.sum() and abs(ne - oe) <= near.sum(), (na, oa, ne, oe)
    assert na > 20000
    xyz, vel, sig, rho = t.particles()
    d0 = sc.params["d0"]
    dx = np.max(np.abs(xyz - st.x)) / d0
    ds = np.sqrt(np.mean((sig - st.sig) ** 2)) / (sc.params["rho0"] * 9.81 * 0.1)
    print("strip window: counts", (na, ne, nb), "oracle", (oa, oe), "dx/d0", dx, "dsig", ds)
    assert dx < 1e-4 and ds < 1e-4
    moved = np.any(st.x != sc.x, axis=1) | np.any(st.sig != sc.sig, axis=1)
    assert (~moved).sum() > 100000
    assert np.array_equal(xyz[~moved], x0[~moved]) and np.array_equal(sig[~moved], s0[~moved])
    for b in range(4):
        F, _ = t.body_wrench(b)
        Fo = st.bodies.wrench[b, :3]
        assert np.linalg.norm(F - Fo) <= 1e-3 * np.linalg.norm(Fo)


@pytest.mark.parametrize("t_delay", [-1.0, 0.00045])
def test_active_skin_agrees_with_per_step_gather(t_delay):
    """Active domains with a Verlet skin keep the working set (gathered with a
    margin beyond the grown boxes) across steps and re-flag it every step; the
    trajectory matches the per-step gather without the skin up to FP32 rounding,
    the flags agree but for particles at a face, terrain never integrated stays
    at its FP32 inputs, and most steps skip the gather and the search."""
    sc = _scene(seed=54, carrier_v=(2.0, 0.0, 0.0), t_delay=t_delay)
    a = crm.from_scene(sc, skin=0.1)
    b = crm.from_scene(sc, skin=0.0)
    a.step(sc.dt, 0)
    b.step(sc.dt, 0)
    x0, _, s0, _ = a.particles()
    xb0, _, sb0, _ = b.particles()
    a.profile_reset()
    n = 60
    a.step(sc.dt, n)
    b.step(sc.dt, n)
    prof = a.profile()
    xa, va, sa, ra = a.particles()
    xb, vb, sb, rb = b.particles()
    d0 = sc.params["d0"]
    assert np.max(np.abs(xa - xb)) < 2e-5 * d0
    assert np.sqrt(np.mean((sa - sb) ** 2)) < 2e-5 * sc.params["rho0"] * 9.81 * 0.1
    na, ne, nb = a.counts()
    ma, me, mb = b.counts()
    st = oracle.State(sc)
    st.run(n)
    near = _near_face(st.x, sc.boxes, st.bodies.pose, sc.params["h"], tol=1e-6)
    assert abs(na - ma) <= near.sum() and abs(ne - me) <= near.sum(), (na, ma, ne, me)
    assert na > 500 and ne > 200
    if t_delay < 0:   # (before t_delay every particle is integrated)
        never = np.all(xb == xb0, axis=1) & np.all(sb == sb0, axis=1)
        assert never.sum() > 1000
        assert np.array_equal(xa[never], x0[never]) and np.array_equal(sa[never], s0[never])
    gathers = prof["launches"]["neighbors"]
    print("active skin: gathers", gathers, "of", n, "steps; counts", (na, ne), (ma, me))
    assert 1 <= gathers < n // 2, prof
    Fa, _ = a.body_wrench(0)
    Fb, _ = b.body_wrench(0)
    assert np.linalg.norm(Fa - Fb) <= 1e-3 * np.linalg.norm(Fb) + 1e-9

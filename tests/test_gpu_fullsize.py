"""Parity at the benchmark's full size: the 120,000-particle wheel bin (65,328 wall
and 5,920 wheel markers) exactly as bench.py builds it and steps it -- the default
Verlet skin, the step graph, the default lanes of the pair kernels -- against the
FP64 oracle on every particle and marker (the oracle is fast enough for that at
this size).

Bars: the rate bars of test_gpu_parity.py with the oracle fed the state the
terrain holds (tests/held.py): |r_gpu - r_oracle| <= 1e-5 S for every particle's
and every marker's every component, with no allowance (measured on a B300: the
worst fluid component at 7.4e-6 S, the worst marker component at 5.0e-6 S, no
kernel-edge exception).  After 1 and 10 graph-replayed steps: the short-horizon
measures of the reduced wheel (position against d0, stress against rho0 g H,
density, the wheel force).
"""
import numpy as np
import pytest

import held
import oracle
import scenes

pytestmark = pytest.mark.gpu

crm = pytest.importorskip("paper_2507_05643_b300")


@pytest.fixture(scope="module")
def bench_scene():
    sc = scenes.wheel_bin()
    assert sc.x.shape[0] == 120000
    return sc


def test_full_size_rates_match_oracle(bench_scene):
    sc = bench_scene.copy()
    t = crm.from_scene(sc)
    edge = held.check_rates("full size", sc, t.eval_rates())
    assert not edge   # every component within the plain bar


def test_full_size_steps_match_oracle(bench_scene):
    """The bench's launch configuration: default skin (the first step searches with
    the skin radius and filters in stage 1), the step graph replayed."""
    sc = bench_scene.copy()
    t = crm.from_scene(sc)
    st = oracle.State(sc)
    d0 = sc.params["d0"]
    sig_scale = sc.params["rho0"] * 9.81 * 0.15
    report = {}
    done = 0
    for k in (1, 10):
        t.step(sc.dt, k - done)
        st.run(k - done)
        done = k
        xyz, vel, sig, rho = t.particles()
        F, _ = t.body_wrench(0)
        Fo = st.bodies.wrench[0, :3]
        report[k] = (float(np.max(np.abs(xyz - st.x)) / d0),
                     float(np.sqrt(np.mean((sig - st.sig) ** 2)) / sig_scale),
                     float(np.max(np.abs(sig - st.sig)) / sig_scale),
                     float(np.max(np.abs(rho - st.rho)) / sc.params["rho0"]),
                     float(np.linalg.norm(F - Fo) / max(np.linalg.norm(Fo), 1e-12)))
    print("full size: max|dx|/d0, rms dsig/(rho0 g H), max|dsig|/(rho0 g H), max|drho|/rho0, "
          "|dF|/|F|:", report)
    dx, ds, dsm, dr, dF = report[1]
    # measured on a B300: 1.9e-7, 1.0e-8, 9.7e-8, 3.6e-8, 3.7e-8 after one step and
    # 9.7e-7, 3.0e-8, 4.3e-7, 3.4e-7, 8.7e-8 after ten
    assert dx < 1e-6 and ds < 1e-7 and dsm < 1e-6 and dr < 1e-6 and dF < 1e-6, report
    dx, ds, dsm, dr, dF = report[10]
    assert dx < 1e-5 and ds < 1e-6 and dsm < 1e-5 and dr < 1e-5 and dF < 1e-6, report
    pose, _ = t.body_state(0)
    assert abs(pose[2] - st.bodies.pose[0, 2]) < 1e-7


def test_full_size_adjoint_matches_the_oracle_adjoint():
    """The differentiable wheel test at its full size (30,000 SPH particles, the
    bench's adjoint scene, skin 0, checkpoints) over 10 steps with a checkpoint
    every 5: every gradient entry against the oracle's own FP64 adjoint, for
    J = mean drawbar pull + mean sinkage over the second half + random weights on
    the final SPH state."""
    from oracle import adjoint as oadj
    sc = scenes.wheel_bin(seed=3, nx=100, ny=30, nz=10)
    sc.params["skin"] = 0.0
    n, every = 10, 5
    t = crm.from_scene(sc)
    t.adjoint_forward(sc.dt, n, every)
    lw = np.zeros((n, 1, 6))
    lw[n // 2:, 0, 0] = 1.0 / (n - n // 2)
    lc = np.zeros((n, 1, 3))
    lc[n // 2:, 0, 2] = -1e3 / (n - n // 2)
    rng = np.random.default_rng(9)
    m = sc.x.shape[0]
    lf = {"x": rng.normal(size=(m, 3)), "u": rng.normal(size=(m, 3)) * 1e-2,
          "sig": rng.normal(size=(m, 6)) * 1e-6, "rho": rng.normal(size=m) * 1e-4}
    g = t.adjoint_backward(lw, lc, lf["x"], lf["u"], lf["sig"], lf["rho"])
    _, _, o = oadj.run_gradients(sc, sc.dt, n, lw, lc, lf, mode="cells")
    errs = {}
    for k, ko in (("xyz", "x"), ("vel", "u"), ("stress", "sig"), ("rho", "rho")):
        a, r = np.asarray(g[k], float).reshape(o[ko].shape), o[ko]
        errs[k] = float(np.linalg.norm(a - r) / np.linalg.norm(r))
    b = np.asarray(g["body"], float)[0]
    for k, sl, r in (("body_c", slice(0, 3), o["body_c"][0]), ("body_v", slice(3, 6), o["body_v"][0]),
                     ("body_w", slice(12, 15), o["body_w"][0])):
        errs[k] = float(np.linalg.norm(b[sl] - r) / np.linalg.norm(r))
    for k in ("E", "nu", "rho0", "mu_s", "cohesion", "av_gamma"):
        errs[k] = abs(float(g["param_grads"][k]) - o["params"][k]) / abs(o["params"][k])
    print("full size adjoint, errors against the oracle adjoint:", errs)
    assert max(errs.values()) < 1e-4, errs


def test_full_ensemble_members_match_oracle():
    """The whole 64-bin ensemble (6.7 M SPH particles) stepped as one batch after
    its autotune, as bench.py runs it -- the persistent form, one launch per stage
    over all 64 bins; the smallest and the largest bin against the oracle stepped
    through the same steps: the autotune's 1 + 3 steps with each of its six
    choices (three lane counts x two cell tiles), then 5 batch steps."""
    import torch
    bins = scenes.ensemble_bins()
    streams = [torch.cuda.Stream() for _ in bins]
    mem = [crm.from_scene(sc, stream=s) for sc, s in zip(bins, streams)]
    dts = [sc.dt for sc in bins]
    batch = crm.Batch(mem, stream=torch.cuda.current_stream())
    batch.autotune(dts, trial_steps=3)
    batch.set_persistent(True)
    batch.step(dts, 5)
    torch.cuda.synchronize()
    sizes = [sc.x.shape[0] for sc in bins]
    report = {}
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        sc = bins[k]
        st = oracle.State(sc)
        st.run(6 * (1 + 3) + 5)
        xyz, vel, sig, rho = mem[k].particles()
        F, _ = mem[k].body_wrench(0)
        Fo = st.bodies.wrench[0, :3]
        report[sizes[k]] = (float(np.max(np.abs(xyz - st.x)) / sc.params["d0"]),
                            float(np.sqrt(np.mean((sig - st.sig) ** 2))
                                  / (sc.params["rho0"] * 9.81 * sc.x[:, 2].max())),
                            float(np.max(np.abs(rho - st.rho)) / sc.params["rho0"]),
                            float(np.linalg.norm(F - Fo) / max(np.linalg.norm(Fo), 1e-12)))
    batch.close()
    print("ensemble members (SPH count: max|dx|/d0, rms dsig/(rho0 g H), max|drho|/rho0, "
          "|dF|/|F|):", report)
    for dx, ds, dr, dF in report.values():
        assert dx < 1e-5 and ds < 1e-6 and dr < 1e-5 and dF < 1e-5, report

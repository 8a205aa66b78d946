"""Seeded synthetic inputs shaped like the paper's terramechanics workloads.

This module is shared by the FP64 oracle tests, the CUDA-path tests and the
benchmark.  It only builds *inputs*: particle lattices, boundary-marker layers,
a grousered wheel, the initial stress state and the material constants.  It
holds none of the method's arithmetic (no kernel, no rates, no return map).

Geometry conventions (paper Sec. 2.4, "Boundary Condition Enforcing Markers"):

* SPH particles sit on a cubic lattice of spacing d0 with centres at
  (i + 1/2) d0 inside the soil block.
* Wall markers continue that lattice outward, N_layers = ceil(2h/d0) layers
  thick (3 for h = 1.2 d0), on the floor and the four sides, up to 0.1 m above
  the free surface.
* Rigid-body markers are given in the body frame; the first layer lies on the
  collision surface and further layers lie inside the body.

Randomness: numpy PCG64 seeded with the workload number; positional jitter
U(-1e-4, 1e-4) m per coordinate on SPH particles only.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

G_EARTH = 9.81

# Activity / body constants shared by the generator and its users.
DOF_X, DOF_Y, DOF_Z = 1, 2, 4
DOF_RX, DOF_RY, DOF_RZ = 8, 16, 32


@dataclasses.dataclass
class Body:
    markers_local: np.ndarray          # (n, 3) body-frame marker coordinates
    pose: np.ndarray                   # (7,) x, y, z, qw, qx, qy, qz
    twist: np.ndarray                  # (6,) vx, vy, vz, wx, wy, wz (world frame)
    mass: float
    dof_mask: int                      # bit k set: linear DOF k integrates (x=1, y=2, z=4);
                                       # bits 3-5: angular DOF k integrates (x=8, y=16, z=32)
    inertia: Optional[np.ndarray] = None   # (3,) principal moments in the body frame
    load: Optional[np.ndarray] = None      # (6,) external force, torque about the centre


@dataclasses.dataclass
class ActiveBox:
    body: int
    half_extents: np.ndarray           # (3,) in the body frame
    offset: np.ndarray                 # (3,) box centre in the body frame


@dataclasses.dataclass
class Scene:
    name: str
    params: Dict[str, object]          # material + numerical constants (SI)
    x: np.ndarray                      # (n, 3) SPH positions
    u: np.ndarray                      # (n, 3) SPH velocities
    sig: np.ndarray                    # (n, 6) stress xx, yy, zz, xy, xz, yz
    rho: np.ndarray                    # (n,)
    fixed: np.ndarray                  # (m, 3) fixed wall markers (world frame)
    bodies: List[Body]
    boxes: List[ActiveBox]
    t_delay: float
    dt: float
    n_steps: int
    domain_min: np.ndarray
    domain_max: np.ndarray

    @property
    def n_fluid(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_markers(self) -> int:
        return int(self.fixed.shape[0] + sum(b.markers_local.shape[0] for b in self.bodies))

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, x=self.x.copy(), u=self.u.copy(), sig=self.sig.copy(), rho=self.rho.copy(),
            fixed=self.fixed.copy(),
            bodies=[dataclasses.replace(b, markers_local=b.markers_local.copy(),
                                        pose=b.pose.copy(), twist=b.twist.copy(),
                                        inertia=None if b.inertia is None else b.inertia.copy(),
                                        load=None if b.load is None else b.load.copy())
                    for b in self.bodies],
            boxes=[dataclasses.replace(bx) for bx in self.boxes],
            params=dict(self.params))


def default_params(d0: float = 0.01, **over) -> Dict[str, object]:
    """Material defaults of the synthetic workloads (rho0 = 1700, E = 1e6, nu = 0.3,
    h = 1.2 d0, gravity -9.81 z, ps_freq 1, unilateral artificial viscosity 0.02)."""
    p: Dict[str, object] = dict(
        rho0=1700.0, E=1.0e6, nu=0.3,
        mu_s=math.tan(math.radians(30.0)), mu_2=None, I0=0.08, grain_d=0.002, cohesion=0.0,
        d0=d0, h=1.2 * d0,
        av_mode=2, av_gamma=0.02, av_xi2_over_h2=0.01,
        gravity=(0.0, 0.0, -G_EARTH),
        ps_freq=1, max_neighbors=96, kernel=0,
    )
    p.update(over)
    if p["mu_2"] is None:
        p["mu_2"] = p["mu_s"]
    return p


def n_layers(h: float, d0: float) -> int:
    """Number of BCE layers, ceil(K h / d0) with K = 2 (paper Sec. 2.4)."""
    return int(math.ceil(2.0 * h / d0 - 1e-9))


def lattice(ni: int, nj: int, nk: int, d0: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Centres (i + 1/2) d0 of an ni x nj x nk block starting at ``origin``; x fastest."""
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    pts = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    return (pts + 0.5) * d0 + np.asarray(origin, dtype=np.float64)


def box_walls(nx: int, ny: int, nz_wall: int, layers: int, d0: float,
              origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Floor + four side walls around an nx x ny interior, ``layers`` thick.

    The walls are the sites of the lattice extended by ``layers`` cells outward in
    x, y and downward in z, up to ``nz_wall`` cells above the floor, minus the
    interior nx x ny x nz_wall sites."""
    full = lattice(nx + 2 * layers, ny + 2 * layers, nz_wall + layers, d0,
                   origin=np.asarray(origin) - layers * d0)
    o = np.asarray(origin)
    rel = (full - o) / d0 - 0.5
    inside = ((rel[:, 0] > -0.5) & (rel[:, 0] < nx - 0.5) & (rel[:, 1] > -0.5)
              & (rel[:, 1] < ny - 0.5) & (rel[:, 2] > -0.5))
    return full[~inside]


def geostatic_stress(z: np.ndarray, surface: float, rho0: float, nu: float,
                     g: float = G_EARTH) -> np.ndarray:
    """Initial lithostatic stress: s_zz = -rho0 g (H - z), s_xx = s_yy = K0 s_zz,
    K0 = nu / (1 - nu); shear zero."""
    szz = -rho0 * g * np.maximum(surface - z, 0.0)
    k0 = nu / (1.0 - nu)
    sig = np.zeros((z.shape[0], 6))
    sig[:, 0] = k0 * szz
    sig[:, 1] = k0 * szz
    sig[:, 2] = szz
    return sig


def quat_about_y(theta: float) -> np.ndarray:
    return np.array([math.cos(theta / 2), 0.0, math.sin(theta / 2), 0.0])


def wheel_markers(radius: float, width: float, d0: float, layers: int = 3,
                  n_grousers: int = 12, grouser_height: float = 0.01,
                  grouser_thickness: float = 0.01) -> np.ndarray:
    """Body-frame markers of a grousered cylindrical wheel, axle along y.

    The rim's first layer lies on the cylinder of the given radius, further
    layers step inward by d0; across the width markers are spaced d0 and include
    both edges.  Each grouser is a plate of the given height and thickness
    standing on the rim, filled with markers at spacing d0."""
    pts = []
    n_w = max(1, int(round(width / d0)) + 1)
    ys = np.linspace(-width / 2, width / 2, n_w)
    for L in range(layers):
        r = radius - L * d0
        n_c = max(8, int(round(2 * math.pi * r / d0)))
        th = 2 * math.pi * np.arange(n_c) / n_c
        for y in ys:
            pts.append(np.stack([r * np.cos(th), np.full(n_c, y), r * np.sin(th)], axis=1))
    n_rad = max(1, int(round(grouser_height / d0)))
    n_tan = max(1, int(round(grouser_thickness / d0)))
    for g in range(n_grousers):
        phi = 2 * math.pi * g / n_grousers
        er = np.array([math.cos(phi), 0.0, math.sin(phi)])
        et = np.array([-math.sin(phi), 0.0, math.cos(phi)])
        for a in range(n_rad):
            rr = radius + (a + 0.5) * grouser_height / n_rad
            for b in range(n_tan):
                tt = ((b + 0.5) / n_tan - 0.5) * grouser_thickness
                for y in ys:
                    pts.append((rr * er + tt * et + np.array([0.0, y, 0.0]))[None, :])
    return np.concatenate(pts, axis=0)


def _jitter(rng: np.random.Generator, x: np.ndarray, amp: float = 1e-4) -> np.ndarray:
    return x + rng.uniform(-amp, amp, size=x.shape)


def settling_block(seed: int = 1, n: int = 20, d0: float = 0.01, box: float = 0.3,
                   jitter: float = 1e-4) -> Scene:
    """Granular block of n^3 SPH particles (spacing d0) centred in x, y on the
    floor of a ``box``-sized container walled by 3 layers of fixed markers.
    Friction 30 deg, cohesion 0, sigma0 = 0, bilateral artificial viscosity
    0.02, dt = 1e-4 s, 200 steps (defaults reproduce the 8,000-particle block)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, mu_s=math.tan(math.radians(30.0)), cohesion=0.0, av_mode=1,
                       av_gamma=0.02)
    nb = int(round(box / d0))
    off = (nb - n) // 2
    x = _jitter(rng, lattice(n, n, n, d0, origin=(off * d0, off * d0, 0.0)), jitter)
    layers = n_layers(p["h"], d0)
    fixed = box_walls(nb, nb, nb, layers, d0)
    m = x.shape[0]
    lo = np.array([-layers * d0 - 2 * p["h"]] * 3)
    hi = np.array([box + layers * d0 + 2 * p["h"]] * 3)
    return Scene("settling_block", p, x, np.zeros((m, 3)), np.zeros((m, 6)),
                 np.full(m, p["rho0"]), fixed, [], [], 0.0, 1e-4, 200, lo, hi)


def wheel_bin(seed: int = 2, nx: int = 200, ny: int = 40, nz: int = 15, d0: float = 0.01,
              wheel_radius: float = 0.2, wheel_width: float = 0.15, n_grousers: int = 12,
              grouser_height: float = 0.01, load_n: float = 100.0, slip: float = 0.3,
              omega: float = 0.8, phi_deg: float = 33.0, cohesion: float = 500.0,
              wheel_x: float = 0.4, dt: float = 5e-5, n_steps: int = 2000,
              jitter: float = 1e-4, geostatic: bool = True, wall_above: float = 0.1,
              active_box: Optional[np.ndarray] = None) -> Scene:
    """Single grousered wheel on a soil bin (defaults: 2.0 x 0.4 x 0.15 m at 0.01 m,
    120,000 particles; wheel r = 0.2 m, width 0.15 m, 12 grousers 0.01 m tall;
    100 N load, slip 0.3, friction 33 deg, cohesion 500 Pa, dt 5e-5 s, 2000 steps).

    The wheel's angular velocity and forward speed are prescribed (speed =
    omega r_g (1 - slip), r_g = r + grouser height), its vertical DOF is free
    with mass load/g, and it starts with the grouser tips on the surface."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, mu_s=math.tan(math.radians(phi_deg)), cohesion=cohesion,
                       av_mode=2, av_gamma=0.02)
    H = nz * d0
    x = _jitter(rng, lattice(nx, ny, nz, d0), jitter)
    layers = n_layers(p["h"], d0)
    nz_wall = nz + int(round(wall_above / d0))
    fixed = box_walls(nx, ny, nz_wall, layers, d0)
    sig = geostatic_stress(x[:, 2], H, p["rho0"], p["nu"]) if geostatic else np.zeros((x.shape[0], 6))
    rg = wheel_radius + grouser_height
    wm = wheel_markers(wheel_radius, wheel_width, d0, layers, n_grousers, grouser_height)
    pose = np.concatenate([[wheel_x, ny * d0 / 2, H + rg], quat_about_y(0.0)])
    v = omega * rg * (1.0 - slip)
    twist = np.array([v, 0.0, 0.0, 0.0, omega, 0.0])
    body = Body(wm, pose, twist, load_n / G_EARTH, DOF_Z)
    boxes = []
    if active_box is not None:
        boxes.append(ActiveBox(0, np.asarray(active_box, dtype=np.float64), np.zeros(3)))
    margin = layers * d0 + 2 * p["h"]
    lo = np.array([-margin, -margin, -margin])
    hi = np.array([nx * d0 + margin, ny * d0 + margin, max(nz_wall * d0, H + 2 * rg) + margin])
    m = x.shape[0]
    return Scene("wheel_bin", p, x, np.zeros((m, 3)), sig, np.full(m, p["rho0"]), fixed,
                 [body], boxes, 0.0, dt, n_steps, lo, hi)


def sphere_markers(radius: float, d0: float, layers: int = 3) -> np.ndarray:
    """Body-frame markers of a sphere: `layers` shells stepping inward by d0 from
    the surface, each covered at about d0 spacing (Fibonacci points)."""
    pts = []
    for L in range(layers):
        r = radius - L * d0
        if r <= 0.0:
            break
        n = max(12, int(round(4 * math.pi * r * r / (d0 * d0))))
        k = np.arange(n) + 0.5
        z = 1.0 - 2.0 * k / n
        phi = math.pi * (1.0 + math.sqrt(5.0)) * k
        rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        pts.append(r * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1))
    return np.concatenate(pts, axis=0)


def sphere_drop(seed: int = 6, nx: int = 30, ny: int = 30, nz: int = 12, d0: float = 0.01,
                radius: float = 0.05, density: float = 7800.0, speed: float = 1.0,
                spin: float = 3.0, phi_deg: float = 30.0, cohesion: float = 0.0,
                dt: float = 5e-5, n_steps: int = 400, jitter: float = 1e-4) -> Scene:
    """A solid sphere dropped onto a granular bed with all six DOFs free (the
    paper's cratering setting of Sec. 4, small): a steel sphere of the given
    radius hits the surface at `speed` with a spin about x, on a geostatic
    nx x ny x nz bed with 3-layer walls.  Inertia of a solid sphere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, mu_s=math.tan(math.radians(phi_deg)), cohesion=cohesion,
                       av_mode=2, av_gamma=0.02)
    H = nz * d0
    x = _jitter(rng, lattice(nx, ny, nz, d0), jitter)
    layers = n_layers(p["h"], d0)
    nz_wall = nz + int(round(0.05 / d0))
    fixed = box_walls(nx, ny, nz_wall, layers, d0)
    sig = geostatic_stress(x[:, 2], H, p["rho0"], p["nu"])
    mass = density * 4.0 / 3.0 * math.pi * radius ** 3
    inertia = np.full(3, 0.4 * mass * radius * radius)
    pose = np.concatenate([[nx * d0 / 2, ny * d0 / 2, H + radius + 0.5 * d0], [1.0, 0.0, 0.0, 0.0]])
    twist = np.array([0.0, 0.0, -speed, spin, 0.0, 0.0])
    body = Body(sphere_markers(radius, d0, layers), pose, twist, mass,
                DOF_X | DOF_Y | DOF_Z | DOF_RX | DOF_RY | DOF_RZ, inertia=inertia,
                load=np.zeros(6))
    margin = layers * d0 + 2 * p["h"]
    lo = np.array([-margin, -margin, -margin])
    hi = np.array([nx * d0 + margin, ny * d0 + margin, max(nz_wall * d0, H + 3 * radius) + margin])
    m = x.shape[0]
    return Scene("sphere_drop", p, x, np.zeros((m, 3)), sig, np.full(m, p["rho0"]), fixed,
                 [body], [], 0.0, dt, n_steps, lo, hi)


def sphere_crater(rho_sphere: float, H: float, seed: int = 8, bed=(0.14, 0.1, 0.1),
                  d0: float = 0.0025, radius: float = 0.0125, dt: float = 5e-5,
                  n_steps: int = 3000, jitter: float = 1e-5) -> Scene:
    """The paper's sphere cratering test (Sec. 4, Sphere Cratering): a sphere of
    radius 0.0125 m and density rho_sphere dropped from height H onto a granular
    bed of density 1510 kg/m^3 and friction mu_s = 0.3 in a 0.14 x 0.1 m
    container, SPH parameters of its table (d0 = 2.5 mm, h = 3.25 mm, bilateral
    artificial viscosity 0.01, cubic spline, dt = 5e-5 s).  Readings where the
    paper is silent: a bed 0.1 m deep at rest under geostatic stress; E = 1e6 Pa,
    nu = 0.3 (the workloads' defaults); mu_2 = mu_s (the rate term needs mu_2,
    which is not given); no cohesion.  The fall itself is not simulated: the
    sphere starts with its lowest point at the surface and the speed sqrt(2 g H)
    it reaches by falling H, its centre free to move vertically only."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, rho0=1510.0, mu_s=0.3, mu_2=0.3, grain_d=0.001, cohesion=0.0,
                       av_mode=1, av_gamma=0.01)
    p["h"] = 0.00325
    nx, ny, nz = (int(round(b / d0)) for b in bed)
    Hb = nz * d0
    x = _jitter(rng, lattice(nx, ny, nz, d0), jitter)
    layers = n_layers(p["h"], d0)
    nz_wall = nz + 4
    fixed = box_walls(nx, ny, nz_wall, layers, d0)
    sig = geostatic_stress(x[:, 2], Hb, p["rho0"], p["nu"])
    mass = rho_sphere * 4.0 / 3.0 * math.pi * radius ** 3
    pose = np.array([nx * d0 / 2, ny * d0 / 2, Hb + radius + 0.5 * d0, 1.0, 0.0, 0.0, 0.0])
    twist = np.array([0.0, 0.0, -math.sqrt(2.0 * G_EARTH * H), 0.0, 0.0, 0.0])
    body = Body(sphere_markers(radius, d0, layers), pose, twist, mass, DOF_Z)
    margin = layers * d0 + 2 * p["h"]
    lo = np.array([-margin, -margin, -margin])
    hi = np.array([nx * d0 + margin, ny * d0 + margin, Hb + 4 * radius + margin])
    m = x.shape[0]
    sc = Scene("sphere_crater", p, x, np.zeros((m, 3)), sig, np.full(m, p["rho0"]), fixed,
               [body], [], 0.0, dt, n_steps, lo, hi)
    return sc


def lattice_only(seed: int, n: int = 12, d0: float = 0.01, jitter: float = 1e-4,
                 random_state: bool = True, **over) -> Scene:
    """An n^3 jittered lattice with random velocities and stresses and no walls
    (used for the momentum-antisymmetry and gradient-consistency checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, **over)
    x = _jitter(rng, lattice(n, n, n, d0), jitter)
    m = x.shape[0]
    if random_state:
        u = rng.uniform(-0.5, 0.5, size=(m, 3))
        sig = rng.uniform(-2000.0, 500.0, size=(m, 6))
        rho = p["rho0"] * (1.0 + rng.uniform(-0.02, 0.02, size=m))
    else:
        u, sig, rho = np.zeros((m, 3)), np.zeros((m, 6)), np.full(m, p["rho0"])
    lo = np.full(3, -4 * p["h"])
    hi = np.full(3, n * d0 + 4 * p["h"])
    return Scene("lattice", p, x, u, sig, rho, np.zeros((0, 3)), [], [], 0.0, 1e-4, 1, lo, hi)


def strip(seed: int = 5, length: float = 1.0e4, width: float = 2.0, depth: float = 0.1,
          d0: float = 0.025, x_window: Optional[tuple] = None, rover_x: float = 5000.0,
          wheel_radius: float = 0.25, wheel_width: float = 0.2, speed: float = 1.0,
          sinkage: float = 0.01, box: float = 1.0, dt: float = 1e-4, n_steps: int = 10000,
          jitter: float = 1e-4) -> Scene:
    """Long terrain strip driven over by a four-wheel kinematic rover with one
    active box per wheel (defaults: 10 km x 2 m x 0.1 m at 0.025 m; wheels
    r = 0.25 m, width 0.2 m, track 1 m, wheelbase 1.5 m, 1 m/s, boxes 1 m).

    ``x_window`` = (x0, x1) keeps only the lattice columns with x0 <= x < x1 (a
    bounded sample of the strip; inactive terrain is frozen, so a window that
    contains every box plus its 2h extension steps identically).  The terrain is
    taken as settled, so the boxes are in force from the first step
    (t_delay = -1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = default_params(d0, mu_s=0.8, cohesion=5000.0, av_mode=2, av_gamma=0.02)
    nx_all, ny, nz = int(round(length / d0)), int(round(width / d0)), int(round(depth / d0))
    i0, i1 = 0, nx_all
    if x_window is not None:
        i0 = max(0, int(math.floor(x_window[0] / d0)))
        i1 = min(nx_all, int(math.ceil(x_window[1] / d0)))
    x = lattice(i1 - i0, ny, nz, d0, origin=(i0 * d0, 0.0, 0.0))
    x = _jitter(rng, x, jitter)
    layers = n_layers(p["h"], d0)
    fl = lattice(i1 - i0, ny, layers, d0, origin=(i0 * d0, 0.0, -layers * d0))
    sig = geostatic_stress(x[:, 2], depth, p["rho0"], p["nu"])
    wm = wheel_markers(wheel_radius, wheel_width, d0, layers, n_grousers=0)
    bodies, boxes = [], []
    zc = depth + wheel_radius - sinkage
    for dx in (0.0, 1.5):
        for yc in (0.5, 1.5):
            pose = np.concatenate([[rover_x + dx, yc, zc], quat_about_y(0.0)])
            twist = np.array([speed, 0.0, 0.0, 0.0, speed / wheel_radius, 0.0])
            bodies.append(Body(wm, pose, twist, 10.0, 0))
            boxes.append(ActiveBox(len(bodies) - 1, np.array([box / 2] * 3), np.zeros(3)))
    margin = layers * d0 + 2 * p["h"]
    lo = np.array([-margin, -margin, -margin])
    hi = np.array([length + margin, width + margin, depth + 2 * wheel_radius + margin])
    m = x.shape[0]
    return Scene("strip", p, x, np.zeros((m, 3)), sig, np.full(m, p["rho0"]), fl,
                 bodies, boxes, -1.0, dt, n_steps, lo, hi)


def ensemble_bins(seed: int = 4, n: int = 64, d0: float = 0.01) -> List[Scene]:
    """The batched ensemble: n single-wheel soil bins of uneven size.  Bin k
    draws u_k ~ U(0, 1) from its own stream (SeedSequence(seed).spawn(n)[k]):
    target particle count 20k + 180k u_k and bin length 0.5 + 1.5 u_k m (size
    and length coupled, so a 0.3 m wide bin keeps a plausible depth of
    round(N / (100 L 30)) layers), then slip U(0.1, 0.7), friction U(25, 40) deg
    and cohesion U(0, 2000) Pa independently; the grousered wheel of wheel_bin
    (r = 0.2 m, width 0.15 m) at 0.2 m from the bin's start."""
    out = []
    for k, ss in enumerate(np.random.SeedSequence(seed).spawn(n)):
        rng = np.random.Generator(np.random.PCG64(ss))
        u = rng.uniform()
        target = 20000 + 180000 * u
        length = 0.5 + 1.5 * u
        nx, ny = int(round(length / d0)), 30
        nz = max(4, int(round(target / (nx * ny))))
        slip = rng.uniform(0.1, 0.7)
        phi = rng.uniform(25.0, 40.0)
        coh = rng.uniform(0.0, 2000.0)
        out.append(wheel_bin(seed=int(ss.generate_state(1)[0] % (2**31)), nx=nx, ny=ny, nz=nz, d0=d0,
                             slip=slip, phi_deg=phi, cohesion=coh, wheel_x=0.3, n_steps=1000))
    return out


def workload(name: str, **kw) -> Scene:
    """Named workloads: 'settling_block' (8,000-particle block), 'wheel_bin'
    (120,000-particle grousered wheel bin), 'diff_wheel_bin' (30,000-particle bin),
    'strip' (10 km active-domain strip)."""
    if name == "settling_block":
        return settling_block(**kw)
    if name == "wheel_bin":
        return wheel_bin(**kw)
    if name == "diff_wheel_bin":
        kw.setdefault("seed", 3)
        return wheel_bin(nx=100, ny=30, nz=10, n_steps=400, wheel_x=0.3, **kw)
    if name == "strip":
        return strip(**kw)
    raise KeyError(name)

"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Each function returns a plain description: lattice size, boundary axes,
relaxation time, body forces, contact constants and a list of particles
(control points in the body frame, weights K_i, sphero radius, density,
position, orientation, velocities).  Both the CUDA path and the CPU oracle
consume these dictionaries through their own constructors.

Shapes follow the paper's workloads made synthetic (there is no dataset):
the single sphere of §3.1 (one control point), the four-control-point
metaball of §3.2, and the randomly shaped metaballs of §4.  Seeds are
2206 + k for workload k = 1..5.  Contact constants and gravities are chosen
here, not taken from the paper (which does not give them); the gravity of a
workload is picked so that the Stokes estimate of its settling speed stays
near 0.02 lattice units per step (low Mach number).
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2206


def _particle(cp, K, x, *, Rs=0.0, density=1.0, q=(1.0, 0.0, 0.0, 0.0), v=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0),
              fixed=0, mass=0.0, inertia=None):
    d = dict(cp=np.asarray(cp, dtype=np.float64).reshape(-1, 3), K=np.asarray(K, dtype=np.float64),
             x=np.asarray(x, dtype=np.float64), Rs=float(Rs), density=float(density),
             q=np.asarray(q, dtype=np.float64), v=np.asarray(v, dtype=np.float64),
             w=np.asarray(w, dtype=np.float64), fixed=int(fixed), mass=float(mass))
    d["inertia"] = None if inertia is None else np.asarray(inertia, dtype=np.float64).reshape(3, 3)
    return d


def _random_quaternion(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def random_metaball(rng, ncp: int, spread: float, K_range=(9.0, 25.0)):
    """Control points uniform in [-spread, spread]^3 and weights uniform in
    K_range (the non-spherical particle of §3.2 made synthetic)."""
    cp = rng.uniform(-spread, spread, (ncp, 3))
    K = rng.uniform(K_range[0], K_range[1], ncp)
    return cp, K


def nominal_radius_metaball(rng, ncp: int, spread: float, radius: float):
    """Control points uniform in [-spread, spread]^3 with weights drawn in
    [0.5, 1.5] and scaled so that sum K = radius^2 (a metaball of one control
    point with that K is the sphere of the given radius, §2.1.2)."""
    cp = rng.uniform(-spread, spread, (ncp, 3))
    w = rng.uniform(0.5, 1.5, ncp)
    K = w / w.sum() * radius * radius
    return cp, K


def bounding_radius(cp, K, Rs=0.0):
    """max |x_i| + sqrt(sum K) + R_s: no point of {M >= 1} lies farther."""
    return float(np.max(np.linalg.norm(cp, axis=1)) + math.sqrt(float(np.sum(K))) + Rs)


def settling_sphere():
    """Workload 1: one control point K = 36 (radius 6) at (15.5, 15.5, 34) in a
    32x32x48 walled box, tau = 0.8, density ratio 2.5, FP64, 300 steps."""
    return dict(name="settling_sphere_32x32x48", nx=32, ny=32, nz=48, periodic=(0, 0, 0), tau=0.8,
                storage="f64", n_sub=100, gravity=(0.0, 0.0, -1e-4), force=(0.0, 0.0, 0.0), steps=300,
                kn=200.0, eta_n=5.0, kt=100.0, eta_t=2.0, mu_s=0.3, c_tol=1e-6,
                particles=[_particle([[0, 0, 0]], [36.0], (15.5, 15.5, 34.0), density=2.5)])


def settling_metaball(tau: float = 0.8, nx: int = 128, ny: int = 128, nz: int = 256, storage: str = "f32",
                      steps: int = 5000):
    """Workload 2: one four-control-point metaball (offsets uniform in +-4,
    K_i uniform in [9, 25], random orientation) settling in a walled
    128x128x256 box, FP32, 5000 steps.  Density ratio 1134/970 as in §3.2."""
    rng = np.random.default_rng(BASE_SEED + 2)
    cp, K = random_metaball(rng, 4, 4.0)
    q = _random_quaternion(rng)
    x = (nx / 2 - 0.5 + rng.uniform(-1, 1), ny / 2 - 0.5 + rng.uniform(-1, 1), nz * 0.78)
    return dict(name=f"settling_metaball_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, periodic=(0, 0, 0), tau=tau,
                storage=storage, n_sub=100, gravity=(0.0, 0.0, -8e-4), force=(0.0, 0.0, 0.0), steps=steps,
                kn=2000.0, eta_n=20.0, kt=1000.0, eta_t=10.0, mu_s=0.3, c_tol=1e-6,
                particles=[_particle(cp, K, x, density=1134.156 / 970.0, q=q, Rs=0.5)])


def multi_particle(nparticles: int = 200, n: int = 256, nz: int | None = None, storage: str = "f32",
                   steps: int = 2000, seed_offset: int = 3):
    """Workload 3: nparticles metaballs of 2-8 control points (offsets
    uniform in +-3, nominal radius uniform in [5, 8], random orientation)
    placed by rejection sampling on bounding spheres with a 2-node gap in an
    n x n x nz box, periodic in x and y, walls in z (as §4's 30-particle run).
    Densities 1200/927 as in §4."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    parts, centres, radii = [], [], []
    Rs = 0.5
    tries = 0
    while len(parts) < nparticles:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place the particles")
        ncp = int(rng.integers(2, 9))
        cp, K = nominal_radius_metaball(rng, ncp, 3.0, rng.uniform(5.0, 8.0))
        b = bounding_radius(cp, K, Rs)
        c = np.array([rng.uniform(0, n), rng.uniform(0, n), rng.uniform(b + 1.5, nz - 1.5 - b)])
        ok = True
        for c2, b2 in zip(centres, radii):
            d = c - c2
            d[:2] -= n * np.round(d[:2] / n)
            if np.linalg.norm(d) < b + b2 + 2.0:
                ok = False
                break
        if not ok:
            continue
        centres.append(c)
        radii.append(b)
        parts.append(_particle(cp, K, c, density=1200.0 / 927.0, q=_random_quaternion(rng), Rs=Rs))
    return dict(name=f"multi_particle_{nparticles}p_{n}x{n}x{nz}", nx=n, ny=n, nz=nz, periodic=(1, 1, 0),
                tau=0.8, storage=storage, n_sub=100, gravity=(0.0, 0.0, -1e-3), force=(0.0, 0.0, 0.0),
                steps=steps, kn=2000.0, eta_n=20.0, kt=1000.0, eta_t=10.0, mu_s=0.3, c_tol=1e-6,
                particles=parts)


def dkt(shape: str = "metaball", storage: str = "f32", steps: int = 8000, tau: float = 0.56):
    """The two-particle settling run of §4 (drafting, kissing, tumbling) in
    lattice units at the paper's resolution (dx = 1 mm, dt = 2e-4 s): a walled
    150 x 150 x 250 box; fluid viscosity 7.55e-5 m^2/s, which is nu = 0.0151
    and tau = 3 nu + 1/2 = 0.5453 -- but at that tau the scheme as read here
    (BGK, VIBB with the non-equilibrium part extrapolated for q > 1/2) diverges
    after about 150 steps, in the FP64 oracle as on the GPU, so the run takes
    tau = 0.56 (nu = 0.02, 1e-4 m^2/s), the lowest value tried that stays
    stable; densities 1200 (particles) and 927 (fluid);
    gravity 9.8 m/s^2 = 3.92e-4 lattice units (applied as the relative gravity
    of §3.1); n_s = dt / dt_DEM = 100.  The particles start at rest 220 and 205
    nodes above the bottom wall, the lower one 2 nodes off the centre line.

    shape "metaball": four control points on a square, (+-2.2, +-2.2, 0), each
    with K = 12.71, the square facing the fall (the paper gives the §3.2
    metaball's volume, 1.648e-6 m^3 = 1648 cells, and elongation 0.84375, not
    its control points; these give a volume of 1648 cells and a thickness /
    width ratio of 0.84).  shape "sphere": one control point with the same
    volume (radius 7.325, K = 53.66).  Sphero radius 0.1 (1e-4 m, as §3.1)."""
    if shape == "metaball":
        a = 2.2
        cp = [[a, a, 0.0], [a, -a, 0.0], [-a, a, 0.0], [-a, -a, 0.0]]
        K = [12.71] * 4
    elif shape == "sphere":
        cp, K = [[0.0, 0.0, 0.0]], [53.66]
    else:
        raise ValueError(f"shape {shape!r}: metaball or sphere")
    nx, ny, nz = 150, 150, 250
    c = (nx - 1) / 2.0
    parts = [_particle(cp, K, (c, c, 220.0 - 0.5), density=1200.0 / 927.0, Rs=0.1),
             _particle(cp, K, (c + 2.0, c, 205.0 - 0.5), density=1200.0 / 927.0, Rs=0.1)]
    return dict(name=f"dkt_{shape}_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, periodic=(0, 0, 0),
                tau=tau, storage=storage, n_sub=100,
                gravity=(0.0, 0.0, -9.8 * 2e-4 ** 2 / 1e-3), force=(0.0, 0.0, 0.0), steps=steps,
                kn=2000.0, eta_n=20.0, kt=1000.0, eta_t=10.0, mu_s=0.3, c_tol=1e-6, particles=parts)


def drag_case(storage: str = "f32", n: int = 48, steps: int = 1000, ncp: int = 4, seed_offset: int = 5):
    """One drag case of the batched sweep: a fixed metaball of ncp control
    points (offsets uniform in +-2.5, nominal radius 6) at the centre of a
    periodic n^3 box, flow driven by a Guo body force 2e-6 along x, tau 0.8,
    fluid at rest initially, 1000 steps (the length of the batched drag sweep)."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    cp, K = nominal_radius_metaball(rng, ncp, 2.5, 6.0)
    c = n / 2.0 - 0.5
    return dict(name=f"drag_{ncp}cp_{n}^3", nx=n, ny=n, nz=n, periodic=(1, 1, 1), tau=0.8, storage=storage, n_sub=0,
                gravity=(0.0, 0.0, 0.0), force=(2e-6, 0.0, 0.0), steps=steps, kn=0.0, eta_n=0.0, kt=0.0, eta_t=0.0,
                mu_s=0.0, c_tol=1e-6,
                particles=[_particle(cp, K, (c + 0.21, c - 0.13, c + 0.07), q=_random_quaternion(rng), fixed=1,
                                     mass=1.0, inertia=np.eye(3))])


def batched_drag(ncases: int = 64, storage: str = "f32", lo: int = 48, hi: int = 128, steps: int = 1000,
                 seed_offset: int = 5):
    """Workload 5, the batched drag sweep: ncases independent periodic cubes
    whose side is uniform on {lo..hi} (reading: uniform on the side length),
    each holding one fixed random metaball of 1-6 control points (offsets
    uniform in +-0.15 side, nominal radius 0.12 side) near its centre, flow
    driven by a Guo body force along x scaled so the Stokes-limit mean speed is
    about the same in every box; tau 0.8; 1000 steps."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    cases = []
    for c in range(ncases):
        n = int(rng.integers(lo, hi + 1))
        ncp = int(rng.integers(1, 7))
        R = 0.12 * n
        cp, K = nominal_radius_metaball(rng, ncp, 0.15 * n / 2.0, R)
        ctr = n / 2.0 - 0.5 + rng.uniform(-0.5, 0.5, 3)
        force = 2e-6 * (48.0 / n) ** 2
        cases.append(dict(name=f"batched_drag_{c}_{n}^3", nx=n, ny=n, nz=n, periodic=(1, 1, 1), tau=0.8,
                          storage=storage, n_sub=0, gravity=(0.0, 0.0, 0.0), force=(force, 0.0, 0.0), steps=steps,
                          kn=0.0, eta_n=0.0, kt=0.0, eta_t=0.0, mu_s=0.0, c_tol=1e-6,
                          particles=[_particle(cp, K, ctr, q=_random_quaternion(rng), fixed=1, mass=1.0,
                                               inertia=np.eye(3))]))
    return cases


def adjoint_case(n: int = 96, ncp: int = 6, T: int = 500, W: int = 100, U: float = 0.02, tau: float = 0.8,
                 seed_offset: int = 4):
    """Workload 4: the drag gradient.  A fixed metaball of ncp control points
    (offsets uniform in +-0.06 n, nominal radius n/9.6 = 10 lu at n = 96) at
    the centre of a periodic n^3 box; fluid started at u = U x (Re = U 2R / nu =
    4 at the defaults), a Guo body force of twice the Stokes drag per unit
    volume along x holds the mean flow; J = mean F_x over the last W of T
    steps.  Control points are given in the world frame (identity
    orientation, x at the box centre)."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    R = n / 9.6
    cp, K = nominal_radius_metaball(rng, ncp, 0.06 * n, R)
    c = np.full(3, n / 2.0 - 0.5) + rng.uniform(-0.3, 0.3, 3)
    nu = (tau - 0.5) / 3.0
    force = 2.0 * 6.0 * np.pi * nu * R * U / float(n) ** 3
    return dict(name=f"adjoint_{ncp}cp_{n}^3", nx=n, ny=n, nz=n, periodic=(1, 1, 1), tau=tau, u0=(U, 0.0, 0.0),
                force=(force, 0.0, 0.0), T=T, W=W, x=c, cp_world=cp + c, K=K)


def empty_box(n: int = 256, storage: str = "f32", periodic=(1, 1, 1)):
    """A lattice with no particles (the sweep's bandwidth ceiling)."""
    return dict(name=f"empty_{n}^3", nx=n, ny=n, nz=n, periodic=periodic, tau=0.8, storage=storage, n_sub=0,
                gravity=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), steps=100, kn=0.0, eta_n=0.0, kt=0.0, eta_t=0.0,
                mu_s=0.0, c_tol=1e-6, particles=[])


def perturbed_populations(rng, Q: int, shape, weights, amp: float = 1e-2, u_amp: float = 0.02):
    """Populations w_i (1 + noise) plus a small random drift, as an arbitrary
    but realistic injected state for one-step comparisons (f[i, z, y, x])."""
    f = np.empty((Q,) + tuple(shape))
    for i in range(Q):
        f[i] = weights[i] * (1.0 + amp * rng.uniform(-1, 1, shape))
    return f

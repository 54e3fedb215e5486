"""Pins of the oracle's contact law (§2.1.1, Eqs. (2)-(3)) against closed forms.

Two spheres of internal radius r = 1000 with skins R_s = 0.01 touch far outside
the lattice box, so no fluid node and no wall takes part.  At this radius the
closest points of Eqs. (7)-(9) err by 3 g^2 / (4 r) for an internal gap g, a
few 1e-8 lu here, so the contact behaves like two flat faces and the textbook
solutions of the spring-dashpot-Coulomb law apply:

- normal dashpot (Eq. (2)): a head-on collision of the linear spring-dashpot
  with the force kept repulsive ends when k_n delta + eta_n d(delta)/dt = 0;
  the relative velocity then leaves with the coefficient of restitution of
  the damped oscillator evaluated at that instant (closed form below), to the
  first order in the sub-step;
- Coulomb cap (Eq. (3)): a solid sphere pressed on a fixed one and launched
  sideways without spin slides with |F_t| = mu_s F_n, decelerates at
  mu_s g_eff, spins up, and ends rolling at 5/7 of its launch speed (angular
  momentum about the contact point is conserved; I = 2/5 m l^2);
- tangential spring in stick (Eq. (3), F_t0 = -k_t xi - eta_t v_t): with the
  rotation locked and mu_s large, the tangential displacement is an
  undamped harmonic oscillator of frequency sqrt(k_t/m) whose spring force is
  -k_t x (xi returns to zero with x), and with eta_t > 0 its amplitude decays
  by exp(-eta_t t / (2 m)).
"""
import numpy as np
import pytest

R_IN = 1000.0
RS = 0.01
BASE = np.array([-5000.0, -5000.0, -5000.0])


def _sphere(oracle_mod, x, v=(0, 0, 0), mass=1.0, inertia=None, fixed=0, density=2.0):
    I = np.eye(3) * (0.4 * mass * R_IN * R_IN) if inertia is None else inertia
    return oracle_mod.make_particle([[0, 0, 0]], [R_IN * R_IN], x, v=v, Rs=RS, density=density, mass=mass,
                                    inertia=I, fixed=fixed)


def _restitution_exact(k, eta, m):
    """Coefficient of restitution of m x'' = -k x - eta x' (x the overlap)
    for a contact that ends when the force k x + eta x' first vanishes."""
    g = eta / (2 * m)
    w0 = np.sqrt(k / m)
    wd = np.sqrt(w0 * w0 - g * g)
    theta = np.pi - np.arctan2(2 * g * wd, w0 * w0 - 2 * g * g)
    t = theta / wd
    return -np.exp(-g * t) * (np.cos(theta) - g / wd * np.sin(theta)), t


def _collide(oracle_mod, ns, k, eta, v0):
    o = oracle_mod.Oracle(4, 4, 4, n_sub=ns, kn=k, eta_n=eta, c_tol=1e-8)
    gap = 0.5 * v0   # the spheres meet after half a step
    a = _sphere(oracle_mod, BASE, v=(0.5 * v0, 0, 0), mass=2.0)
    b = _sphere(oracle_mod, BASE + [2 * R_IN + 2 * RS + gap, 0, 0], v=(-0.5 * v0, 0, 0), mass=2.0)
    o.set_particles([a, b])
    steps = 0
    while steps < 200:
        o.step(1)
        steps += 1
        st = o.get_particles()
        if steps > 3 and not np.abs(o.contact_forces()[0]).max() > 0:
            break
    st = o.get_particles()
    return (st[1]["v"][0] - st[0]["v"][0]) / v0


@pytest.mark.parametrize("zeta", [0.05, 0.3])
def test_normal_dashpot_restitution(oracle_mod, zeta):
    k, m_eff, v0 = 1.0, 1.0, 0.01     # two masses of 2
    eta = 2 * zeta * np.sqrt(k * m_eff)
    e_exact, t_contact = _restitution_exact(k, eta, m_eff)
    assert 2.0 < t_contact < 4.0       # the contact lasts a few LBM steps
    e50 = _collide(oracle_mod, 50, k, eta, v0)
    e200 = _collide(oracle_mod, 200, k, eta, v0)
    # the force switches on with a jump of eta v0 at the first sub-step in
    # contact: first order in h = 1/n_s
    assert abs(e50 - e_exact) < 2 * eta / m_eff / 50
    assert abs(e200 - e_exact) < 2 * eta / m_eff / 200
    assert abs(e200 - e_exact) < abs(e50 - e_exact) or abs(e200 - e_exact) < 1e-5
    # without the clamp the law would give the plain damped-oscillator value
    w0, g = np.sqrt(k / m_eff), eta / (2 * m_eff)
    e_unclamped = np.exp(-np.pi * g / np.sqrt(w0 * w0 - g * g))
    assert abs(e200 - e_unclamped) > 10 * abs(e200 - e_exact)


def _pressed_pair(oracle_mod, ns, g_eff, kn, eta_n, kt, eta_t, mu, v0, inertia=None, mass=1.0):
    """Sphere B resting on the fixed sphere A under the relative gravity g_eff
    (density 2: (1 - rho0/rho_s) g = g/2), placed at the static overlap
    m g_eff / k_n (found with the oracle's own pair geometry, an input)."""
    grav = (0.0, 0.0, -2.0 * g_eff)
    delta0 = mass * g_eff / kn
    o = oracle_mod.Oracle(4, 4, 4, n_sub=ns, kn=kn, eta_n=eta_n, kt=kt, eta_t=eta_t, mu_s=mu, c_tol=1e-8,
                          gravity=grav)
    lo, hi = 2 * R_IN, 2 * R_IN + 2 * RS
    for _ in range(60):   # bisection on the centre distance for delta = delta0
        mid = 0.5 * (lo + hi)
        o.set_particles([_sphere(oracle_mod, BASE, fixed=1), _sphere(oracle_mod, BASE + [0, 0, mid])])
        hit, delta, *_ = o.pair_geometry(0, 1)
        if hit and delta > delta0:
            lo = mid
        else:
            hi = mid
    D = 0.5 * (lo + hi)
    ell = R_IN + RS - 0.5 * delta0   # lever arm: the middle of the overlap
    I = np.eye(3) * (0.4 * mass * ell * ell) if inertia is None else inertia
    o.set_particles([_sphere(oracle_mod, BASE, fixed=1),
                     _sphere(oracle_mod, BASE + [0, 0, D], v=(v0, 0, 0), mass=mass, inertia=I)])
    return o


def test_coulomb_cap_while_sliding(oracle_mod):
    """Without tangential damping the reported load is the spring alone,
    which the cap resets to exactly mu_s F_n at every sub-step of sliding."""
    g_eff, mu, v0 = 1e-3, 0.3, 0.01
    o = _pressed_pair(oracle_mod, 100, g_eff, 1.0, 2.0, 1.0, 0.0, mu, v0)
    t_slide = 2 * v0 / (7 * mu * g_eff)
    for step in range(1, int(t_slide) - 1):
        o.step(1)
        F, _ = o.contact_forces()
        # (the cap was set with the normal force of the last sub-step)
        assert abs(np.hypot(F[1, 0], F[1, 1]) / F[1, 2] / mu - 1) < 2e-4
        assert F[1, 0] < 0          # against the sliding direction
        # deceleration mu g_eff (F_n = m g_eff at the static overlap)
        assert abs(o.get_particles()[1]["v"][0] - (v0 - mu * g_eff * step)) < 5e-4 * v0


def test_coulomb_sliding_then_rolling(oracle_mod):
    """The lower sphere is curved (radius 1000): once rolling, the upper one
    slowly rolls off it under gravity (about 1e-4 of v0 by step 25), so the
    end state is taken a few steps after the slip stops."""
    g_eff, mu, v0 = 1e-3, 0.3, 0.01
    kn, kt = 1.0, 1.0
    o = _pressed_pair(oracle_mod, 100, g_eff, kn, 2.0, kt, 1.0, mu, v0)
    t_slide = 2 * v0 / (7 * mu * g_eff)      # sliding ends when v = w l
    assert 8 < t_slide < 11
    vs = []
    for step in range(1, 26):
        o.step(1)
        vs.append(o.get_particles()[1]["v"][0])
    # while sliding: deceleration mu g_eff
    for t in range(2, int(t_slide) - 1):
        assert abs(vs[t - 1] - (v0 - mu * g_eff * t)) < 5e-4 * v0
    # then rolling without slip at 5/7 of the launch speed
    st = o.get_particles()[1]
    ell = R_IN + RS - 0.5 * g_eff / kn
    assert abs(st["v"][0] / v0 - 5.0 / 7.0) < 3e-4
    assert abs(st["w"][1] * ell - st["v"][0]) < 1e-4 * v0
    # a sign error in the friction torque would spin the sphere the other way
    assert st["w"][1] > 0


@pytest.mark.parametrize("eta_t", [0.0, 0.1])
def test_tangential_spring_in_stick(oracle_mod, eta_t):
    g_eff, kn, kt, m, v0 = 1e-3, 1.0, 0.25, 1.0, 1e-3
    locked = np.eye(3) * 1e30     # no rotation: the contact point moves with the centre
    o = _pressed_pair(oracle_mod, 100, g_eff, kn, 2.0, kt, eta_t, 100.0, v0, inertia=locked, mass=m)
    x0 = o.get_particles()[1]["x"][0]
    wt = np.sqrt(kt / m)
    g = eta_t / (2 * m)
    wd = np.sqrt(wt * wt - g * g)
    err_x = err_F = 0.0
    for step in range(1, 40):
        o.step(1)
        st = o.get_particles()[1]
        x = st["x"][0] - x0
        exact = v0 / wd * np.exp(-g * step) * np.sin(wd * step)
        F, _ = o.contact_forces()
        err_x = max(err_x, abs(x - exact))
        # spring force -k_t xi with xi = x, plus the dashpot on the contact velocity
        err_F = max(err_F, abs(F[1, 0] - (-kt * x - eta_t * st["v"][0])))
    amp = v0 / wt
    # second order in h = 1e-2 for the spring; the dashpot sees the
    # half-step velocity, first order: h eta_t / (2 m) relative
    assert err_x < (1e-4 + 2 * g / 100) * amp
    # (xi is kept in the tangent plane, which tilts by x / (2 r) as the sphere moves)
    assert err_F < 1e-5 * kt * amp

"""Pins for the oracle's free DEM (Section 2.2, Eqs. 4-11), independent of the oracle itself:
closed forms for sphere contacts (single-centre metaballs are spheres, and the sphero-metaball
of a sphere is that sphere), conservation laws, a separately integrated contact ODE for the
coefficient of restitution, the static overlap under gravity, the 5/7 rolling law, the exact
free-fall sequence of symplectic Euler, and torque-free spin."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2308_05007_gb300 import inputs as I


def _spheres(centers, ks, dims=(48, 48, 48), walls=0, Rs=None, velocity=None, spin=None, kn=200.0,
             eta_n=0.0, kt=0.0, eta_t=0.0, mu_s=0.0, gravity=(0.0, 0.0, 0.0), substeps=20, density=2.0):
    """Single-centre particles (spheres of radius sqrt(k)); returns the oracle, masses, inertias."""
    P = len(ks)
    mb = I.Metaballs(
        center_offsets=np.arange(P + 1, dtype=np.int32),
        centers_body=np.zeros((P, 3), np.float32),
        k=np.asarray(ks, np.float32),
        origin=np.asarray(centers, np.float64).reshape(P, 3),
        amplitude=np.zeros((P, 3)), period=np.zeros(P), phase=np.zeros(P), omega=np.zeros((P, 3)))
    dem = I.Dem(density=density,
                sphere_radius=np.asarray(Rs if Rs is not None else [0.25 * math.sqrt(k) for k in ks], float),
                velocity=None if velocity is None else np.asarray(velocity, float),
                spin=None if spin is None else np.asarray(spin, float),
                kn=kn, eta_n=eta_n, kt=kt, eta_t=eta_t, mu_s=mu_s, gravity=gravity, substeps=substeps,
                hydro=0)
    w = I.Workload(name="dem_spheres", dims=dims, tau=0.8, D=0.0, seed=0, wall_mask=walls, metaballs=mb,
                   dem=dem)
    o = Oracle.from_workload(w, seed_walkers=False)
    mp = o.dem_mass()
    return o, mp[:, 0], mp[:, 4:10]


def test_mass_properties_of_a_sphere():
    """Sampled at h = 1/4: a sphere of radius 5 and density 2 has mass (4/3) pi r^3 rho and inertia
    (2/5) m r^2 to the sampling error (~1e-3), its centre of mass at the centre exactly (the grid
    and the inside test are symmetric), and no products of inertia."""
    o, m, Ib = _spheres([[20.0, 21.0, 22.0]], [25.0], density=2.0)
    mp = o.dem_mass()[0]
    assert m[0] == pytest.approx(2.0 * 4.0 / 3.0 * math.pi * 125.0, rel=5e-3)
    np.testing.assert_array_equal(mp[1:4], [0.0, 0.0, 0.0])
    for a in range(3):
        assert Ib[0, a] == pytest.approx(0.4 * m[0] * 25.0, rel=5e-3)
    np.testing.assert_array_equal(Ib[0, 3:], [0.0, 0.0, 0.0])


def test_mass_properties_of_a_cluster():
    """Two centres: equal weights put the centre of mass midway (exactly, by symmetry); a heavier
    one pulls it towards itself. The shape keeps its world position when the body frame moves to
    the centre of mass (to binary32 rounding of the control points)."""
    def two(k2, sep=3.0):
        mb = I.Metaballs(center_offsets=np.array([0, 2], np.int32),
                         centers_body=np.array([[-sep, 0.0, 0.0], [sep, 0.0, 0.0]], np.float32),
                         k=np.array([16.0, k2], np.float32), origin=np.array([[24.0, 24.0, 24.0]]),
                         amplitude=np.zeros((1, 3)), period=np.zeros(1), phase=np.zeros(1),
                         omega=np.zeros((1, 3)))
        dem = I.Dem(density=1.5, sphere_radius=np.array([1.0]), hydro=0)
        w = I.Workload(name="two", dims=(48, 48, 48), tau=0.8, D=0.0, seed=0, metaballs=mb)
        o = Oracle.from_workload(w, seed_walkers=False)
        probe = np.array([24.0 + sep + 3.9, 24.0, 24.0])
        before = o.metaball(0, probe)[0]
        o.set_dem(dem)
        after = o.metaball(0, probe)[0]
        return o.dem_mass()[0], before, after
    eq, b0, a0 = two(16.0)
    assert eq[1] == 0.0 and eq[2] == 0.0 and eq[3] == 0.0
    assert abs(a0 - b0) < 1e-6 * b0
    hv, b1, a1 = two(36.0)
    assert 0.5 < hv[1] < 3.0 and hv[2] == 0.0 and hv[3] == 0.0
    assert abs(a1 - b1) < 1e-6 * b1
    assert hv[0] > eq[0]


def test_pair_geometry_of_two_spheres_is_exact():
    """Two single-centre particles (radii 6 and 4) overlapping by 0.1 along an oblique line:
    Eqs. 7-9 give the overlap exactly, the normal along the line of centres (from 0 towards 1)
    and the contact point in the middle of the overlap, for any sphere radius R_s."""
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    o0 = np.array([20.0, 17.0, 15.0])
    o1 = o0 + 9.9 * u
    for Rs in ([1.5, 1.0], [3.0, 0.5], [0.2, 2.5]):
        o, _, _ = _spheres([o0, o1], [36.0, 16.0], Rs=Rs)
        g = o.dem_pair_geom(0, 1)
        assert g["delta"] == pytest.approx(0.1, abs=1e-9)
        np.testing.assert_allclose(g["n"], u, atol=1e-10)
        np.testing.assert_allclose(g["xcp"], o0 + (6.0 - 0.05) * u, atol=1e-9)
        np.testing.assert_allclose(g["xc0"], o0 + (6.0 - Rs[0]) * u, atol=1e-9)
        np.testing.assert_allclose(g["xc1"], o1 - (4.0 - Rs[1]) * u, atol=1e-9)
        # the stationary point of f0 + f1 lies on the line of centres
        r = g["xm"] - o0
        assert np.linalg.norm(r - (r @ u) * u) < 1e-9


def test_pair_geometry_across_a_periodic_face():
    """The same pair split by the periodic x face: the minimum image gives the same contact."""
    u = np.array([1.0, 0.0, 0.0])
    o0 = np.array([45.0, 20.0, 20.0])
    o1 = o0 + 9.9 * u - np.array([48.0, 0.0, 0.0])
    o, _, _ = _spheres([o0, o1], [36.0, 16.0], Rs=[1.5, 1.0])
    g = o.dem_pair_geom(0, 1)
    assert g["delta"] == pytest.approx(0.1, abs=1e-9)
    np.testing.assert_allclose(g["n"], u, atol=1e-10)


def test_wall_geometry_of_a_sphere_is_exact():
    """A sphere of radius 5 at height 4.7 over the z = 0 face overlaps it by 0.3; one at 4.8 below
    the z = 48 face by 0.2. Normal into the box, contact point delta/2 inside it (Eq. 11)."""
    o, _, _ = _spheres([[20.0, 21.0, 4.7], [30.0, 25.0, 43.2]], [25.0, 25.0], walls=4, Rs=[1.0, 2.0])
    lo = o.dem_wall_geom(0, 4)
    assert lo["delta"] == pytest.approx(0.3, abs=1e-9)
    np.testing.assert_allclose(lo["n"], [0, 0, 1], atol=0)
    np.testing.assert_allclose(lo["xcw"], [20.0, 21.0, 0.0], atol=1e-9)
    np.testing.assert_allclose(lo["xcp"], [20.0, 21.0, 0.15], atol=1e-9)
    np.testing.assert_allclose(lo["xcm"], [20.0, 21.0, 4.7 - 4.0], atol=1e-9)
    hi = o.dem_wall_geom(1, 5)
    assert hi["delta"] == pytest.approx(0.2, abs=1e-9)
    np.testing.assert_allclose(hi["n"], [0, 0, -1], atol=0)


def test_pair_geometry_is_symmetric_for_clusters():
    """Multi-centre particles: exchanging the two gives the same overlap and the opposite normal."""
    w = I.dem_box(n_particles=2, seed=5)
    mb = w.metaballs
    # move particle 1 next to particle 0
    d = np.array([1.0, 0.4, -0.3]) / np.linalg.norm([1.0, 0.4, -0.3])
    o = Oracle.from_workload(w, seed_walkers=False)
    st = o.particle_state()
    for gap in (3.0, 4.0, 5.0):
        st[1, :3] = st[0, :3] + gap * d
        o.set_particle_state(st)
        a, b = o.dem_pair_geom(0, 1), o.dem_pair_geom(1, 0)
        assert a["delta"] == pytest.approx(b["delta"], abs=1e-9)
        np.testing.assert_allclose(a["n"], -b["n"], atol=1e-9)
        assert abs(np.linalg.norm(a["n"]) - 1.0) < 1e-12
    del mb


def test_free_fall_is_the_symplectic_euler_sequence():
    """No contact: after k DEM steps v = k dt g and z = z0 + dt^2 g k (k + 1) / 2 exactly (to
    rounding), and the spin-free orientation stays the identity."""
    g = -3e-4
    o, _, _ = _spheres([[24.0, 24.0, 30.0]], [9.0], gravity=(0.0, 0.0, g), substeps=8)
    o.dem_advance(5)
    st = o.particle_state()[0]
    k, dt = 40, 1.0 / 8
    assert st[9] == pytest.approx(k * dt * g, rel=1e-13)
    assert st[2] == pytest.approx(30.0 + dt * dt * g * k * (k + 1) / 2, abs=1e-12)
    np.testing.assert_array_equal(st[3:7], [1.0, 0.0, 0.0, 0.0])


def _head_on(m_ratio_k=(36.0, 16.0), v=(0.03, -0.02), eta_n=0.0, kn=200.0, substeps=40, steps=400):
    u = np.array([0.0, 0.6, 0.8])
    o0 = np.array([24.0, 14.0, 14.0])
    o1 = o0 + 10.4 * u
    o, mass, _ = _spheres([o0, o1], list(m_ratio_k), Rs=[1.0, 1.0], velocity=[v[0] * u, v[1] * u],
                          kn=kn, eta_n=eta_n, substeps=substeps)
    p_hist, e_hist, contact = [], [], False
    for _ in range(steps):
        o.dem_advance(1)
        st = o.particle_state()
        p_hist.append(mass[0] * st[0, 7:10] + mass[1] * st[1, 7:10])
        e_hist.append(0.5 * mass[0] * st[0, 7:10] @ st[0, 7:10] + 0.5 * mass[1] * st[1, 7:10] @ st[1, 7:10])
        gap = np.linalg.norm(st[1, :3] - st[0, :3]) - 10.0
        contact |= gap < 0
    st = o.particle_state()
    return o, mass, u, np.array(p_hist), np.array(e_hist), st, contact


def test_elastic_collision_conserves_momentum_and_energy():
    """Head-on elastic collision of unequal spheres: momentum is conserved to rounding at every
    step (equal and opposite pair forces), and the final velocities are the elastic ones to the
    integrator's O(dt) error."""
    o, mass, u, P, E, st, contact = _head_on()
    assert contact
    p0 = mass[0] * 0.03 * u + mass[1] * (-0.02) * u
    assert np.abs(P - p0).max() <= 1e-13 * np.abs(p0).max() * 10
    v0, v1 = 0.03, -0.02
    m0, m1 = mass
    v0f = ((m0 - m1) * v0 + 2 * m1 * v1) / (m0 + m1)
    v1f = ((m1 - m0) * v1 + 2 * m0 * v0) / (m0 + m1)
    assert st[0, 7:10] @ u == pytest.approx(v0f, rel=2e-3)
    assert st[1, 7:10] @ u == pytest.approx(v1f, rel=2e-3)
    assert E[-1] == pytest.approx(E[0], rel=2e-3)


def _restitution_ode(m_eff, kn, eta, v_in, dt=1e-4):
    """Brute-force RK4 of the 1D contact: overlap x, m_eff x'' = -max(0, kn x + eta x')."""
    def acc(x, v):
        return -max(0.0, kn * x + eta * v) / m_eff
    x, v = 0.0, v_in
    while True:
        k1x, k1v = v, acc(x, v)
        k2x, k2v = v + 0.5 * dt * k1v, acc(x + 0.5 * dt * k1x, v + 0.5 * dt * k1v)
        k3x, k3v = v + 0.5 * dt * k2v, acc(x + 0.5 * dt * k2x, v + 0.5 * dt * k2v)
        k4x, k4v = v + dt * k3v, acc(x + dt * k3x, v + dt * k3v)
        x += dt / 6 * (k1x + 2 * k2x + 2 * k3x + k4x)
        v += dt / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
        if x < 0.0 and v < 0.0:
            return -v / v_in


def test_damped_collision_restitution_matches_the_contact_ode():
    eta = 15.0
    o, mass, u, P, E, st, contact = _head_on(eta_n=eta, substeps=200, steps=300)
    m_eff = mass[0] * mass[1] / (mass[0] + mass[1])
    e_ode = _restitution_ode(m_eff, 200.0, eta, 0.05)
    rel_out = (st[0, 7:10] - st[1, 7:10]) @ u
    e_dem = -rel_out / 0.05
    assert 0.2 < e_ode < 0.95
    assert e_dem == pytest.approx(e_ode, abs=2e-3)


def test_resting_overlap_on_the_floor_is_mg_over_kn():
    g, kn = -4e-4, 200.0
    o, mass, _ = _spheres([[24.0, 24.0, 4.95]], [25.0], walls=4, gravity=(0.0, 0.0, g), kn=kn, eta_n=60.0,
                          substeps=20)
    o.dem_advance(1200)   # the start overlap of 0.05 bounces it for ~500 steps
    st = o.particle_state()[0]
    delta = 5.0 - st[2]
    assert delta == pytest.approx(-mass[0] * g / kn, rel=1e-6)
    assert abs(st[9]) < 1e-9


def test_sliding_sphere_ends_rolling_at_five_sevenths():
    """A solid sphere launched without spin along a floor with Coulomb friction slides, then
    rolls without slipping at 5/7 of its launch speed (I = 2/5 m r^2)."""
    g, kn, v0 = -1e-3, 400.0, 0.04
    rest = 4.0 - 0.5 * (0.0)  # centre height; the overlap settles at m g / kn
    o, mass, inertia = _spheres([[10.0, 24.0, rest]], [16.0], walls=4, gravity=(0.0, 0.0, g), kn=kn,
                                eta_n=40.0, kt=200.0, eta_t=10.0, mu_s=0.3, velocity=[[v0, 0.0, 0.0]],
                                substeps=20)
    assert inertia[0, 1] == pytest.approx(0.4 * mass[0] * 16.0, rel=5e-3)
    o.dem_advance(800)
    st = o.particle_state()[0]
    vx, wy = st[7], st[11]
    r = 4.0 - 0.5 * (-mass[0] * g / kn)   # lever arm: centre to the contact point
    # sliding ends in rolling: m v0 = m v + I w / r with v = w r (angular momentum about the
    # contact line), i.e. v = v0 / (1 + I / (m r^2)); 5/7 v0 for I = 2/5 m r^2
    assert vx == pytest.approx(v0 / (1.0 + inertia[0, 1] / (mass[0] * r * r)), rel=1e-2)
    assert vx == pytest.approx(5.0 / 7.0 * v0, rel=1.5e-2)
    assert vx - wy * r == pytest.approx(0.0, abs=2e-3 * v0)


def test_torque_free_isotropic_spin():
    """An isotropic body spins at constant angular velocity (the gyroscopic term vanishes
    exactly) and its orientation turns by |w| t about w, to the first-order integrator's error."""
    w = np.array([0.004, -0.006, 0.012])
    o, _, _ = _spheres([[24.0, 24.0, 24.0]], [9.0], spin=[w], substeps=10)
    o.dem_advance(100)
    st = o.particle_state()[0]
    # the sampled inertia is isotropic to ~1e-3, so the gyroscopic term nearly vanishes
    np.testing.assert_allclose(st[10:13], w, rtol=0, atol=1e-5 * np.linalg.norm(w))
    ang = np.linalg.norm(w) * 100
    ax = w / np.linalg.norm(w)
    want = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax])
    np.testing.assert_allclose(st[3:7], want, atol=5e-4)
    assert abs(np.linalg.norm(st[3:7]) - 1.0) < 1e-14


def test_periodic_many_body_momentum_is_conserved():
    """Frictional, damped collisions among several clusters in a periodic box, no gravity, no
    walls, fluid force off: total momentum is conserved to rounding."""
    w = I.dem_box(dims=(30, 28, 26), n_particles=5, seed=3, speed=0.08, gravity=(0.0, 0.0, 0.0), hydro=0)
    w = I.with_(w, wall_mask=0)
    o = Oracle.from_workload(w, seed_walkers=False)
    m = o.dem_mass()[:, 0]
    p0 = (m[:, None] * o.particle_state()[:, 7:10]).sum(0)
    touched = False
    for _ in range(400):
        o.dem_advance(1)
        st = o.particle_state()
        v = st[:, 7:10]
        touched |= bool(np.abs(v - w.dem.velocity).max() > 1e-6)
        p = (m[:, None] * v).sum(0)
        assert np.abs(p - p0).max() <= 1e-12 * np.abs(m[:, None] * w.dem.velocity).sum()
    assert touched


def test_fluid_drags_free_particles():
    """Coupled step (Eq. 4 with F^e, T^e from the partially saturated cells): particles at rest
    in a fluid driven along x by a body force pick up +x velocity; fluid mass is conserved."""
    w = I.dem_box(dims=(24, 22, 30), n_particles=2, seed=2, speed=0.0, gravity=(0.0, 0.0, 0.0), hydro=1,
                  n_walkers=200)
    w = I.with_(w, body_force=(2e-5, 0.0, 0.0))
    w.dem.velocity[:] = 0.0
    w.dem.spin[:] = 0.0
    o = Oracle.from_workload(w)
    o.step(30)
    st = o.particle_state()
    assert (st[:, 7] > 1e-6).all(), st[:, 7:10]
    assert np.abs(st[:, 8:10]).max() < 0.5 * st[:, 7].min()
    mass = o.density().sum()
    assert mass == pytest.approx(o.n_cells * 1.0, rel=1e-12)


def test_contact_law_normal_clamp_coulomb_limit_and_spring_projection():
    """The contact law on its own. At rest the force on i is -k_n delta n (away from j). It is
    never attractive: a fast separation gives exactly zero. The tangential force is capped at
    mu_s F_n, and the spring then holds the Coulomb force. The spring is first projected onto
    the current tangent plane, so no normal component survives a turning contact."""
    kn, eta_n, kt, eta_t, mu_s = 200.0, 30.0, 80.0, 2.0, 0.3
    o, _, _ = _spheres([[10.0, 24.0, 24.0], [30.0, 24.0, 24.0]], [9.0, 9.0], kn=kn, eta_n=eta_n, kt=kt,
                       eta_t=eta_t, mu_s=mu_s)
    n = np.array([0.0, 0.0, 1.0])
    z3 = np.zeros(3)
    F, xi = o.dem_contact_force(0.05, n, z3, z3, 0.1, z3)
    np.testing.assert_allclose(F, -kn * 0.05 * n, rtol=1e-15)
    assert np.all(xi == 0.0)
    # approaching at 0.1 adds damping; separating at 1.0 would pull (200*0.05 - 30*1 < 0): zero
    F, _ = o.dem_contact_force(0.05, n, np.array([0, 0, 0.1]), z3, 0.1, z3)
    np.testing.assert_allclose(F, -(kn * 0.05 + eta_n * 0.1) * n, rtol=1e-14)
    F, _ = o.dem_contact_force(0.05, n, z3, np.array([0, 0, 1.0]), 0.1, z3)
    assert np.all(F == 0.0)
    # sliding: j moves along x relative to i; unsaturated, then saturated at mu_s F_n
    vj = np.array([0.01, 0.0, 0.0])
    F, xi = o.dem_contact_force(0.05, n, z3, vj, 0.1, z3)
    Fn = kn * 0.05
    np.testing.assert_allclose(xi, vj * 0.1, rtol=1e-15)
    np.testing.assert_allclose(F, kt * xi + eta_t * vj - Fn * n, rtol=1e-14)
    assert np.hypot(F[0], F[1]) < mu_s * Fn
    vj = np.array([0.5, 0.0, 0.0])
    F, xi = o.dem_contact_force(0.05, n, z3, vj, 0.1, np.array([0.2, 0.0, 0.0]))
    assert np.hypot(F[0], F[1]) == pytest.approx(mu_s * Fn, rel=1e-14) and F[0] > 0
    np.testing.assert_allclose(kt * xi + eta_t * vj, [mu_s * Fn, 0.0, 0.0], rtol=1e-13, atol=1e-15)
    # a spring left from an earlier normal loses its component along the new normal
    n2 = np.array([0.0, math.sqrt(0.5), math.sqrt(0.5)])
    _, xi = o.dem_contact_force(0.05, n2, z3, z3, 0.1, np.array([0.01, 0.02, -0.03]))
    assert abs(xi @ n2) < 1e-17
    np.testing.assert_allclose(xi, [0.01, 0.025, -0.025], rtol=1e-14)


def _dumbbell(spin, substeps=10, q0=None):
    """One free two-centre particle (anisotropic inertia), no gravity, no walls, fluid force off."""
    mb = I.Metaballs(center_offsets=np.array([0, 2], np.int32),
                     centers_body=np.array([[-2.5, 0.5, 0.0], [2.5, -0.5, 0.3]], np.float32),
                     k=np.array([9.0, 6.0], np.float32), origin=np.array([[24.0, 24.0, 24.0]]),
                     amplitude=np.zeros((1, 3)), period=np.zeros(1), phase=np.zeros(1), omega=np.zeros((1, 3)))
    dem = I.Dem(density=2.0, sphere_radius=np.array([0.5]), spin=np.asarray([spin], float),
                velocity=np.zeros((1, 3)), substeps=substeps, hydro=0)
    w = I.Workload(name="dumbbell", dims=(48, 48, 48), tau=0.8, D=0.0, seed=0, metaballs=mb, dem=dem)
    o = Oracle.from_workload(w, seed_walkers=False)
    if q0 is not None:
        st = o.particle_state()
        st[0, 3:7] = q0
        o.set_particle_state(st)
    return o


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_torque_free_anisotropic_body_keeps_its_angular_momentum():
    """Euler's equations without torque: the world angular momentum R I_b R^T w stays fixed while
    w itself precesses (the gyroscopic term at work). Explicit Euler drifts by O(dt) only."""
    o = _dumbbell([0.004, 0.009, -0.006])
    Ib6 = o.dem_mass()[0, 4:10]
    Ib = np.array([[Ib6[0], Ib6[3], Ib6[4]], [Ib6[3], Ib6[1], Ib6[5]], [Ib6[4], Ib6[5], Ib6[2]]])
    assert np.ptp(np.linalg.eigvalsh(Ib)) > 0.2 * np.linalg.eigvalsh(Ib).max()   # anisotropic

    def L_world():
        st = o.particle_state()[0]
        R = _rot(st[3:7])
        return R @ Ib @ R.T @ st[10:13], st[10:13].copy()

    L0, w0 = L_world()
    o.dem_advance(400)
    L1, w1 = L_world()
    assert np.linalg.norm(w1 - w0) > 0.05 * np.linalg.norm(w0)       # w does precess
    assert np.linalg.norm(L1 - L0) < 2e-3 * np.linalg.norm(L0)


def test_spin_turns_the_body_in_the_world_frame():
    """The spin is a world-frame angular velocity: from orientation R0 a constant spin w about z
    gives R(t) = R_z(|w| t) R0, not R0 R_z(|w| t). A sphere keeps its spin (isotropic)."""
    q0 = np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0])   # 90 degrees about x
    w = 0.01
    o, _, _ = _spheres([[24.0, 24.0, 24.0]], [9.0], spin=[[0.0, 0.0, w]], substeps=10)
    st = o.particle_state()
    st[0, 3:7] = q0
    o.set_particle_state(st)
    o.dem_advance(150)
    R = _rot(o.particle_state()[0, 3:7])
    a = w * 150
    Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    np.testing.assert_allclose(R, Rz @ _rot(q0), atol=2e-3)
    assert np.abs(R - _rot(q0) @ Rz).max() > 0.5


def test_oblique_frictional_collision_conserves_angular_momentum():
    """Two spheres meet off-centre with friction, no gravity, no walls, fluid force off. The pair
    forces are equal and opposite at one contact point, so the total angular momentum
    sum_p (x_p x m_p v_p + I_p w_p) is conserved. With symplectic Euler and isotropic inertia the
    step keeps it exactly, to rounding. Friction turns some of the orbital part into spin."""
    o, m, Ib = _spheres([[20.0, 24.0, 24.0], [27.0, 25.8, 24.0]], [9.0, 9.0],
                        velocity=[[0.06, 0.0, 0.0], [-0.06, 0.0, 0.0]], kn=200.0, eta_n=5.0, kt=60.0,
                        eta_t=1.0, mu_s=0.4, substeps=20)

    def L():
        st = o.particle_state()
        tot = np.zeros(3)
        for p in range(2):
            tot += np.cross(st[p, 0:3], m[p] * st[p, 7:10]) + Ib[p, 0:3] * st[p, 10:13]
        return tot, st

    L0, _ = L()
    o.dem_advance(120)
    L1, st = L()
    assert np.linalg.norm(st[:, 10:13]) > 1e-4                   # friction spun them up
    scale = m[0] * 0.06 * 1.8
    assert np.linalg.norm(L1 - L0) < 1e-9 * scale, (L0, L1)
    np.testing.assert_array_equal(Ib[:, 0], Ib[:, 1])            # isotropic sampled inertia
    np.testing.assert_array_equal(Ib[:, 0], Ib[:, 2])

"""Pins for the oracle's IBB coupling (Section 2.4.3: interpolated bounce-back, Eqs. 23-25;
Galilean-invariant momentum exchange; refilling, Eqs. 26-27), independent of the oracle itself:
node classes against a brute force, closed-form ray-sphere intersections for q, the link
formula's special cases, an exact momentum balance for a resting particle, the rest state, and
Galilean invariance of the force."""
import numpy as np
import pytest

from oracle.oracle import Oracle, ibb_link, lattice
from paper_2308_05007_gb300 import inputs as I


def _sphere_workload(n=24, center=(12.3, 11.7, 12.1), k=36.0, F=(0.0, 0.0, 0.0), tau=0.8,
                     velocity=(0.0, 0.0, 0.0), particle_velocity=None):
    mb = I.single_sphere(center, k=k)
    if particle_velocity is not None:
        # a sinusoid whose velocity is particle_velocity at t = 0 and stays within 1e-6 of it
        # over the first steps: period 1e6, amplitude v T / (2 pi)
        T = 1e6
        mb.period[:] = T
        mb.phase[:] = 0.0
        mb.amplitude[0] = np.asarray(particle_velocity) * T / (2 * np.pi)
    return I.Workload(name="ibb_sphere", dims=(n, n, n), tau=tau, D=0.0, seed=0, q=15,
                      body_force=F, init_velocity=velocity, metaballs=mb, coupling=1, steps=1)


def test_node_classes_are_the_binary32_inside_test_at_cell_centres():
    """A node is solid when Eq. 3 of some particle reaches 1 at the cell centre, decided in
    binary32 as r2 = (dx dx + dy dy) + dz dz, f = k / r2; where two particles overlap, the lower
    index owns the node. Brute force over every cell of two overlapping spheres."""
    n = 20
    centres = np.array([[8.0, 10.2, 9.7], [11.0, 9.9, 10.3]])
    ks = np.array([6.25, 5.3], np.float32)
    mb = I.Metaballs(center_offsets=np.array([0, 1, 2], np.int32), centers_body=np.zeros((2, 3), np.float32),
                     k=ks, origin=centres, amplitude=np.zeros((2, 3)), period=np.zeros(2),
                     phase=np.zeros(2), omega=np.zeros((2, 3)))
    w = I.Workload(name="ibb_two", dims=(n, n, n), tau=0.8, D=0.0, seed=0, q=15, metaballs=mb,
                   coupling=1, steps=1)
    o = Oracle.from_workload(w, seed_walkers=False)
    node = o.nodes(0)
    idx = np.arange(n ** 3)
    x = (np.stack([idx % n, idx // n % n, idx // (n * n)], 1) + 0.5).astype(np.float32)
    want = np.zeros(n ** 3, np.int32)
    for p in (1, 0):                       # the lower index written last wins
        d = x - centres[p].astype(np.float32)
        r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.float32)
        r2 = (r2 + d[:, 2] * d[:, 2]).astype(np.float32)
        with np.errstate(divide="ignore"):
            inside = (ks[p] / r2).astype(np.float32) >= np.float32(1.0)
        want[inside] = p + 1
    assert np.array_equal(node, want)
    both = [c for c in range(n ** 3) if node[c] == 1
            and np.sum((x[c] - centres[1]) ** 2) < ks[1]]
    assert len(both) > 5                     # the overlap holds nodes, and particle 0 owns them


def test_q_is_the_ray_sphere_intersection():
    """For one centre f = k/r^2, the surface f = 1 is the sphere r = sqrt(k); q along every link
    from a fluid node into a solid node is the smaller root of |x + s e - c|^2 = k."""
    w = _sphere_workload()
    o = Oracle.from_workload(w, seed_walkers=False)
    e, _ = lattice(w.q)
    node = o.nodes(0)
    n = w.dims[0]
    c = np.array(w.metaballs.origin[0])
    R2 = w.metaballs.k[0]
    checked = 0
    for cell in np.where(node == 0)[0]:
        ijk = np.array([cell % n, (cell // n) % n, cell // (n * n)])
        x = ijk + 0.5
        for m in range(1, w.q):
            s = (ijk + e[m]) % n
            if node[(s[2] * n + s[1]) * n + s[0]] == 0:
                continue
            d = x - c
            a, b, cc = e[m] @ e[m], 2 * d @ e[m], d @ d - R2
            s_exact = (-b - np.sqrt(b * b - 4 * a * cc)) / (2 * a)
            assert 0.0 < s_exact <= 1.0
            assert abs(o.ibb_q(0, 0, ijk, e[m]) - s_exact) <= 1e-5, (ijk, e[m])
            checked += 1
    assert checked > 500


def test_link_formula_special_cases():
    q = 15
    e, w = lattice(q)
    i = int(np.where((e == [1, 0, 0]).all(1))[0][0])
    ip = int(np.where((e == [-1, 0, 0]).all(1))[0][0])
    rho = 1.02
    u = np.array([0.03, -0.01, 0.02])
    Gp = 0.13

    def feq(m, r, v):
        eu = e[m] @ v
        return w[m] * r * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * v @ v)

    # q = 1/2 with one velocity everywhere: the moving-wall bounce-back G+_i' + 6 w rho e_i.u_w
    assert ibb_link(q, i, 0.5, rho, u, u, u, Gp) == pytest.approx(Gp + 6 * w[ip] * rho * (e[i] @ u), abs=1e-15)
    # q = 1: u_d* = u_d** = u_w, so the equilibrium part is taken at the wall velocity
    uf, uff, uw = np.array([0.01, 0.0, 0.0]), np.array([0.02, 0.01, 0.0]), np.array([0.0, 0.0, 0.04])
    want = feq(ip, rho, uw) + Gp - feq(ip, rho, uf) + 6 * w[ip] * rho * (e[i] @ uw)
    assert ibb_link(q, i, 1.0, rho, uf, uff, uw, Gp) == pytest.approx(want, abs=1e-15)
    # the two branches of u_d* meet at q = 1/2
    lo = ibb_link(q, i, 0.5, rho, uf, uff, uw, Gp)
    hi = ibb_link(q, i, 0.5 + 1e-12, rho, uf, uff, uw, Gp)
    assert abs(lo - hi) < 1e-11
    # q -> 0: u_d* = u_ff, u_d** = u_ff, so the equilibrium part is taken at u_ff
    want0 = feq(ip, rho, uff) + Gp - feq(ip, rho, uf) + 6 * w[ip] * rho * (e[i] @ uw)
    assert ibb_link(q, i, 1e-14, rho, uf, uff, uw, Gp) == pytest.approx(want0, abs=1e-12)


def _fluid_momentum(o, q):
    e, _ = lattice(q)
    f = o.populations()
    fluid = o.nodes() == 0
    return (e.T.astype(float) @ f[:, fluid]).sum(1), int(fluid.sum())


def test_resting_particle_momentum_balance_is_exact():
    """A particle at rest: the fluid's momentum changes by the body force on its nodes minus the
    momentum exchanged with the particle, P(t+1) - P(t) = N_f F - F_p, to rounding."""
    F = np.array([2e-5, -1e-5, 5e-6])
    w = _sphere_workload(F=tuple(F))
    o = Oracle.from_workload(w, seed_walkers=False)
    o.step_fluid(3)
    for _ in range(3):
        P0, nf = _fluid_momentum(o, w.q)
        o.step_fluid(1)
        P1, nf1 = _fluid_momentum(o, w.q)
        Fp = o.forces()[0, :3]
        assert nf == nf1
        # rounding of the two sums over nf nodes x Q populations of size < 1
        np.testing.assert_allclose(P1 - P0, nf * F - Fp, rtol=0, atol=2 * nf * w.q * 2.0 ** -52)
    assert np.linalg.norm(Fp) > 1e-3 * nf * np.linalg.norm(F)   # the particle does take force


def test_rest_state_is_kept():
    w = _sphere_workload()
    o = Oracle.from_workload(w, seed_walkers=False)
    o.step_fluid(4)
    assert np.abs(o.velocity()).max() < 1e-15
    assert np.abs(o.forces()).max() < 1e-14


def test_force_is_galilean_invariant():
    """Fluid and particle translating together at U: the momentum exchange (Galilean-invariant
    form) sees no force beyond rounding, IBB keeps the stream uniform, and refilled nodes start
    at the stream's velocity; the same particle held at rest in the same stream feels the drag."""
    U = (0.04, 0.0, 0.0)
    moving = Oracle.from_workload(_sphere_workload(velocity=U, particle_velocity=U), seed_walkers=False)
    held = Oracle.from_workload(_sphere_workload(velocity=U), seed_walkers=False)
    nodes0 = moving.nodes(0)
    moving.step_fluid(4)
    held.step_fluid(4)
    assert (moving.nodes(4) != nodes0).sum() > 10   # nodes were covered and uncovered (refilled)
    f_moving = np.linalg.norm(moving.forces()[0, :3])
    f_held = np.linalg.norm(held.forces()[0, :3])
    assert f_held > 1.0
    assert f_moving < 1e-6 * f_held, (f_moving, f_held)
    # the stream around the co-moving particle stays uniform (to the particle's 1e-6 drift from
    # constant velocity over these steps, and rounding)
    u = moving.velocity().reshape(-1, 3)
    assert np.abs(u - np.array(U)).max() < 1e-9


def _overlapping_pair(U, q=15, n=28):
    """Two k = 36 spheres (radius 6) eight cells apart along x, overlapping in a lens; both
    translate at U x (a sinusoid of period 1e6 whose velocity at t = 0 is U), in a stream that
    starts at the equilibrium of velocity U x."""
    T = 1e6
    mb = I.Metaballs(center_offsets=np.array([0, 1, 2], np.int32), centers_body=np.zeros((2, 3), np.float32),
                     k=np.array([36.0, 36.0], np.float32), origin=np.array([[10.3, 14.2, 13.9], [18.3, 14.2, 13.9]]),
                     amplitude=np.array([[U * T / (2 * np.pi), 0.0, 0.0]] * 2), period=np.full(2, T),
                     phase=np.zeros(2), omega=np.zeros((2, 3)))
    return I.Workload(name="ibb_pair", dims=(n, n, n), tau=0.8, D=0.0, seed=0, q=q, metaballs=mb, coupling=1,
                      init_velocity=(U, 0.0, 0.0), steps=1)


@pytest.mark.parametrize("q", [15, 19])
def test_overlapping_particles_force_is_galilean_invariant(q):
    """Each particle of an overlapping pair owns an open piece of the union's surface: lattice
    lines through the lens enter at one particle and leave at the other, so neither particle's
    links come in entry/exit pairs. A stream and both particles translating together at U along
    the line of centres must exert the same force along U on each particle as the same pair at
    rest in still fluid (the pressure on its open surface): in the frame of the moving surface
    nothing crosses it. With the equilibrium at U on both sides of every link and u_f = u_ff =
    u_w = U, Eq. 24 gives G_i = G+_i' + 6 w rho e_i.U, and the Galilean-invariant exchange
    (e_i' - u_w) G+_i' - (e_i - u_w) G_i changes along U by w rho U^2 e_x (9 e_x^2 - 9) = 0 per
    link, exactly. The plain exchange e_i' G+_i' - e_i G_i instead picks up the convective flux
    rho U^2 A through the lens's cross-section A (about 66 lattice lines here), 0.1 at U = 0.04."""
    rest = Oracle.from_workload(_overlapping_pair(0.0, q), seed_walkers=False)
    moving = Oracle.from_workload(_overlapping_pair(0.04, q), seed_walkers=False)
    assert np.array_equal(rest.nodes(0), moving.nodes(0))
    node = rest.nodes(0)
    assert (node == 1).sum() > 100 and (node == 2).sum() > 100
    rest.step_fluid(1)
    moving.step_fluid(1)
    fr, fm = rest.forces()[:, :3], moving.forces()[:, :3]
    # the open surfaces feel the lattice pressure rho c_s^2 over the lens cross-section, opposite
    # on the two particles (about 66/3 along x)
    assert fr[0, 0] > 15.0 and fr[1, 0] < -15.0
    assert fr[0, 0] + fr[1, 0] == pytest.approx(0.0, abs=1e-9)
    np.testing.assert_allclose(fm[:, 0], fr[:, 0], rtol=0, atol=1e-12)

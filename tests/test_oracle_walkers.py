"""Pins of the oracle's random-walk step (Eq. 2), the velocity interpolation of Section 2.4.1,
Algorithms 1 and 2, the Dirichlet refill, walls, binning (Eq. 16), moments and seeding."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle.oracle import Oracle
from paper_2308_05007_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_trilinear_reproduces_affine_fields():
    dims = (9, 8, 7)
    o = Oracle(dims)
    A = np.array([[0.01, -0.02, 0.005], [0.003, 0.0, -0.01], [0.02, 0.01, 0.004]])
    b = np.array([0.1, -0.2, 0.05])
    idx = np.arange(np.prod(dims))
    xn = np.stack([idx % 9, idx // 9 % 8, idx // 72], 1) + 0.5
    o.set_velocity(xn @ A.T + b)
    rng = np.random.default_rng(0)
    for _ in range(100):
        x = rng.uniform(0.5, np.array(dims) - 0.5)   # inside the node lattice: no wrap
        assert np.allclose(o.trilinear(x), A @ x + b, atol=1e-14)
    # periodic wrap: between node n-1 and node 0 the value interpolates across the face
    u = np.zeros((len(idx), 3))
    u[:, 0] = np.where(xn[:, 0] == 0.5, 1.0, 0.0)
    o.set_velocity(u)
    assert o.trilinear([8.75, 3.5, 3.5])[0] == pytest.approx(0.25, abs=1e-15)
    assert o.trilinear([0.25, 3.5, 3.5])[0] == pytest.approx(0.75, abs=1e-15)


def test_trilinear_wall_layer_goes_linearly_to_zero():
    dims = (4, 4, 6)
    o = Oracle(dims, wall_mask=4)
    o.set_velocity(np.tile([0.3, 0.0, 0.0], (96, 1)))
    for z, expect in ((0.0, 0.0), (0.125, 0.075), (0.25, 0.15), (0.5, 0.3), (3.0, 0.3),
                      (5.5, 0.3), (5.75, 0.15), (6.0, 0.0)):
        assert o.trilinear([1.3, 2.2, z])[0] == pytest.approx(expect, abs=1e-15)


def test_mean_square_displacement_is_6Dt():
    """Quiescent fluid, no particles: <|x - x0|^2> = 6 D t (Eq. 2 with u = 0)."""
    D, T, N = 0.03, 60, 20000
    o = Oracle((16, 16, 16), D=D, seed=4)
    o.set_walkers(np.random.default_rng(1).uniform(0, 16, (N, 3)))
    o.step(T)
    m = o.moments()
    msd = m[4:7].sum() + (m[1:4] ** 2).sum()
    assert msd == pytest.approx(6 * D * T, rel=4 * np.sqrt(2 / (3 * N)))
    for a in range(3):
        assert m[4 + a] == pytest.approx(2 * D * T, rel=5 * np.sqrt(2 / N))


def test_reflecting_walls_keep_a_uniform_distribution_uniform():
    """Between two no-slip walls in quiescent fluid, specular reflection leaves a uniform
    distribution uniform: the reflected Gaussian step is symmetric. A wall that clamped or
    absorbed walkers would heap them at the faces. Once mixed across the gap, the z
    displacement variance of independent uniform start and end points is H^2/6."""
    D, H, T, N = 0.2, 8, 300, 20000
    o = Oracle((6, 6, H), D=D, seed=9, wall_mask=4)
    o.set_walkers(np.random.default_rng(2).uniform([0, 0, 0], [6, 6, H], (N, 3)))
    o.step(T)
    x, x0 = o.walkers()
    z = x[:, 2]
    assert z.min() >= 0.0 and z.max() <= H
    counts = np.histogram(z, bins=2 * H, range=(0, H))[0]
    assert stats.chisquare(counts).pvalue > 1e-3, counts
    assert counts[0] / counts.mean() == pytest.approx(1, abs=0.1)
    assert counts[-1] / counts.mean() == pytest.approx(1, abs=0.1)
    var_z = np.mean((z - x0[:, 2]) ** 2)
    assert var_z == pytest.approx(H * H / 6, rel=0.04)
    # the periodic axes still diffuse freely: 2 D t per axis
    for a in (0, 1):
        assert np.mean((x[:, a] - x0[:, a]) ** 2) == pytest.approx(2 * D * T, rel=5 * np.sqrt(2 / N))


def _golden_lattice():
    g = json.load(open(os.path.join(GOLDEN, "point_source_section3_1.json")))
    n = int(round(g["domain_m"] / g["dx_m"]))
    D = g["D_m2_per_s"] * g["dt_s"] / g["dx_m"] ** 2
    u = np.array(g["u_m_per_s"]) * g["dt_s"] / g["dx_m"]
    return g, n, D, u


def test_golden_point_source_parameters_in_lattice_units():
    g, n, D, u = _golden_lattice()
    assert n == 100 and D == pytest.approx(0.2) and np.allclose(u, [0.2, 0, 0])


@pytest.mark.parametrize("flow", [False, True])
def test_point_source_matches_eqs_31_and_34(flow):
    """Section 3.1: a point source spreads as the Gaussian of Eq. 31 (no flow) or Eq. 34
    (uniform flow u); per axis, x - x0 - u t ~ N(0, 2 D t). The paper's parameters in lattice
    units (D = 0.2, u = 0.2) with fewer walkers (the statistics scale with sqrt(N)). Positions
    are unwrapped, so a 20^3 periodic box stands in for the 100^3 one."""
    g, n, D, u = _golden_lattice()
    u = u if flow else np.zeros(3)
    N, T = 20000, 50
    n = 20
    o = Oracle((n, n, n), tau=1.0, D=D, seed=8, init_velocity=tuple(u))
    o.set_walkers(np.full((N, 3), n / 2.0))
    o.step(T)
    x, x0 = o.walkers()
    d = x - x0 - u * T
    for a in range(3):
        res = stats.kstest(d[:, a] / np.sqrt(2 * D * T), "norm")
        assert res.pvalue > 1e-4, (a, res)
        assert abs(d[:, a].mean()) < 5 * np.sqrt(2 * D * T / N)
    # concentration per Eq. 32 (walkers per unit volume) integrates to N (mass conservation)
    assert o.concentration().sum() == N


def _taylor_dispersion(u_nodes, H, D, m=400000):
    """Taylor's long-time dispersion for any profile u(z) between no-flux walls at 0 and H:
    D_eff = D + <G^2> / D with G(z) = int_0^z (u - U) ds and U the mean of u over the channel.
    Here u is the profile the walkers see: linear between the node values at z = k + 1/2 and zero
    on the wall planes. For the parabola it gives D [1 + (2/105) (U h / D)^2]."""
    zn = np.concatenate([[0.0], np.arange(H) + 0.5, [float(H)]])
    un = np.concatenate([[0.0], u_nodes, [0.0]])
    z = (np.arange(m) + 0.5) * H / m
    u = np.interp(z, zn, un)
    G = np.cumsum(u - u.mean()) * (H / m)
    return D + (G * G).mean() / D


def test_taylor_aris_dispersion_in_plane_poiseuille():
    """Walkers in steady force-driven flow between walls at z = 0, H = 2h: the long-time
    streamwise dispersion is D [1 + (2/105) (U h / D)^2] with U the mean velocity (Taylor-Aris
    for a plane channel). Checks the LBM -> walker coupling as a whole. 1e5 walkers, slope of
    the variance between t = 600 (about 5 relaxation times h^2 / (pi^2 D) of the cross-channel
    mode) and t = 1800: statistical error about 0.4%. The closed form holds to 3%; Taylor's
    general formula on the profile the walkers actually interpolate (piecewise linear, 1% below
    the parabola's value at this resolution) holds to 1.5%."""
    H, D, F = 8, 0.05, 2e-3
    tau = 0.5 + np.sqrt(3 / 16)
    nu = (tau - 0.5) / 3
    o = Oracle((2, 2, H), q=15, tau=tau, D=D, seed=21, wall_mask=4, body_force=(F, 0, 0))
    o.step_fluid(3000)
    U = o.velocity()[:, 0].mean()
    # mean of the exact parabola F z (H - z) / (2 nu) over the nodes z = k + 1/2
    assert U == pytest.approx(F * (H * H / 6.0 + 1.0 / 12.0) / (2 * nu), rel=1e-6)
    u_nodes = o.velocity()[:, 0].reshape(H, 2, 2).mean((1, 2))
    N = 100_000
    rng = np.random.default_rng(5)
    o.set_walkers(np.stack([rng.uniform(0, 2, N), rng.uniform(0, 2, N), rng.uniform(0, H, N)], 1))
    o.step(600)
    v1 = o.moments()[4]
    o.step(1200)
    v2 = o.moments()[4]
    Deff = (v2 - v1) / (2 * 1200)
    Pe = U * (H / 2) / D
    expect = D * (1 + 2.0 / 105.0 * Pe * Pe)
    assert Pe > 3 and expect > 1.5 * D   # the flow term is 40% of the dispersion
    assert Deff == pytest.approx(expect, rel=0.03), (Deff, expect, D)
    assert Deff == pytest.approx(_taylor_dispersion(u_nodes, H, D), rel=0.015)
    # walkers never leave the channel
    x, _ = o.walkers()
    assert x[:, 2].min() >= 0.0 and x[:, 2].max() <= H


def _sphere(c=(10.0, 10.0, 10.0), k=16.0, dims=(20, 20, 20)):
    o = Oracle(dims)
    o.set_metaballs(I.single_sphere(c, k))
    return o


def test_algorithm1_finds_the_surface_of_a_sphere():
    """Algorithm 1 on a chord that enters a sphere of radius 4: the result is on the segment
    and |f - 1| < 1e-3, i.e. within 5e-4 r of the sphere."""
    o = _sphere()
    rng = np.random.default_rng(2)
    c = np.array([10.0, 10.0, 10.0])
    for _ in range(50):
        a = c + rng.normal(size=3) * 3
        a = c + (a - c) / np.linalg.norm(a - c) * rng.uniform(4.05, 6.0)
        b = c + rng.normal(size=3) * 1.0
        b = c + (b - c) / np.linalg.norm(b - c) * rng.uniform(0.5, 3.9)
        ok, xi = o.bisect(0, a, b)
        assert ok
        f, _ = o.metaball(0, xi)
        assert abs(f - 1.0) < 1e-3
        # analytic crossing of the segment a + s (b - a) with |x - c| = 4
        dv, w = b - a, a - c
        qa, qb, qc = dv @ dv, 2 * dv @ w, w @ w - 16.0
        s = (-qb - np.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
        # f = 16 / r^2 within 1e-3 of 1 puts r within 5.0e-4 r of 4; the crossing is on the chord
        assert abs(np.linalg.norm(xi - c) - 4.0) < 4.0 * 5.01e-4
        along = (xi - a) @ dv / (dv @ dv)
        assert 0.0 < along < 1.0
        assert np.linalg.norm(xi - (a + along * dv)) < 1e-12
        # and near the analytic crossing (the chord may meet the surface at a glancing angle)
        assert abs(along - s) * np.linalg.norm(dv) < 0.05


def test_algorithm1_reports_failure_without_a_bracket():
    o = _sphere()
    ok, _ = o.bisect(0, [1.0, 1.0, 1.0], [2.0, 1.0, 1.0])   # both ends outside
    assert not ok


def test_algorithm2_is_a_mirror_about_the_normal():
    """Eqs. 18-22: t_r = t_i - 2 (t_i . n) n with the unit normal of a sphere (radial)."""
    o = _sphere()
    c = np.array([10.0, 10.0, 10.0])
    rng = np.random.default_rng(3)
    for _ in range(30):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        xint = c + 4.0 * nrm
        xf = xint + rng.normal(size=3) * 0.3
        xnew = o.reflect(0, xint, xf)
        ti, tr = xf - xint, xnew - xint
        assert np.linalg.norm(tr) == pytest.approx(np.linalg.norm(ti), rel=1e-12)
        assert tr @ nrm == pytest.approx(-(ti @ nrm), abs=1e-12)
        assert np.allclose(tr - (tr @ nrm) * nrm, ti - (ti @ nrm) * nrm, atol=1e-12)


def test_refill_places_walker_outside_near_the_surface():
    """Type II (Section 2.4.2): a walker found inside is pushed out along the gradient and
    placed in a ball of radius sqrt(2 D dt) about the surface point."""
    o = Oracle((20, 20, 20), D=0.02)
    o.set_metaballs(I.single_sphere((10.0, 10.0, 10.0), 16.0))
    rng = np.random.default_rng(4)
    R = np.sqrt(2 * 0.02)
    for i in range(100):
        x = 10.0 + rng.normal(size=3) * 1.2
        assert o.inside(x) == 0
        ok, xn = o.refill(0, x, i)
        assert ok and o.inside(xn) == -1
        r = np.linalg.norm(xn - 10.0)
        assert 4.0 * (1 - 2.6e-4) <= r <= 4.0 + R + 2e-3
        # pushed out along the gradient: same side as the start
        assert (xn - 10.0) @ (x - 10.0) > 0


def test_refill_is_uniform_in_the_ball_about_the_surface_point():
    """The refilled walker lies in the ball of radius R = sqrt(2 D dt) about the surface point x_s
    on the push-out ray. Points that fall inside the particle are mirrored across the tangent
    plane through x_s, which keeps their distance to x_s. So |x_new - x_s| / R has the radial
    law of a uniform ball, P(r <= s) = s^3."""
    D = 0.5
    R = math.sqrt(2 * D)
    o = Oracle((20, 20, 20), D=D)
    o.set_metaballs(I.single_sphere((10.0, 10.0, 10.0), 16.0))
    u = np.array([0.48, -0.6, 0.64])
    x = 10.0 + 2.5 * u                       # inside, radius 2.5; the ray leaves along u
    xo = 10.0 + 4.5 * u                      # first outside point of the steps 1/2, 1, 2
    assert o.inside(10.0 + 3.5 * u) == 0 and o.inside(xo) == -1
    ok, xs = o.bisect(0, xo, x)
    assert ok
    r = []
    for i in range(4000):
        ok, xn = o.refill(0, x, i)
        assert ok and o.inside(xn) == -1
        r.append(np.linalg.norm(xn - xs) / R)
    r = np.array(r)
    assert r.max() <= 1.0 + 1e-12
    assert stats.kstest(r, lambda s: np.clip(s, 0, 1) ** 3).pvalue > 1e-3


def test_walker_type_rules_on_exact_moves():
    """Section 2.4.2's rules on proposals made exact (D = 0, uniform u), against particle A
    (radius 2) and a small particle B placed on the point where a reflection off A lands:
    - type I, out to out: moves to x_p + u;
    - type III, in to out: moves freely to x_p + u;
    - type IV, out to in: Algorithm 1, then Algorithm 2 gives the new point;
    - type IV whose reflected point lies inside a particle or beyond a wall: the walker stays at
      x_p ("multiple reflections ... returned to their original location")."""
    u = np.array([1.2, 0.0, 0.0])
    hit = np.array([7.3, 10.9, 10.0])                 # reaches A at x ~ 8.21, reflects to ~(8.04, 11.13)

    def world(with_b):
        cB = [8.04394206, 11.12982447, 10.0] if with_b else [3.0, 3.0, 3.0]
        mb = I.Metaballs(center_offsets=np.array([0, 1, 2], np.int32), centers_body=np.zeros((2, 3), np.float32),
                         k=np.array([4.0, 0.09], np.float32), origin=np.array([[10.0, 10.0, 10.0], cB]),
                         amplitude=np.zeros((2, 3)), period=np.zeros(2), phase=np.zeros(2), omega=np.zeros((2, 3)))
        o = Oracle((20, 20, 20), D=0.0)
        o.set_metaballs(mb)
        o.set_velocity(np.tile(u, (8000, 1)))
        return o

    o = world(False)
    ok, xi = o.bisect(0, hit, hit + u, 1)
    assert ok
    tr = o.reflect(0, xi, hit + u, 1)
    x = np.array([[3.0, 15.0, 15.0], [11.3, 10.0, 10.0], hit])   # types I, III, IV
    assert [o.inside(v, 1) for v in x] == [-1, 0, -1] and o.inside(x[1] + u, 1) == -1
    out = o.walkers_advance(x, np.arange(3, dtype=np.uint32))
    np.testing.assert_array_equal(out[0], x[0] + u)
    np.testing.assert_array_equal(out[1], x[1] + u)
    np.testing.assert_array_equal(out[2], tr)
    assert o.inside(tr, 1) == -1 and np.linalg.norm(tr - hit) > 0.5
    c = o.counters()
    assert (c["type_I"], c["type_II"], c["type_III"], c["type_IV"]) == (1, 0, 1, 1)
    # the same hit with particle B sitting on the reflected point: back to x_p
    o = world(True)
    assert o.inside(tr, 1) == 1 and o.inside(hit, 1) == -1 and o.inside(hit + u, 1) == 0
    out = o.walkers_advance(hit[None, :], np.array([2], np.uint32))
    np.testing.assert_array_equal(out[0], hit)
    # a reflection off a sphere near the z = 0 wall that would end beyond the wall: back to x_p
    o = Oracle((20, 20, 12), D=0.0, wall_mask=4)
    o.set_metaballs(I.single_sphere((10.0, 10.0, 2.0), 4.0))
    o.set_velocity(np.tile([0.7, 0.0, 0.0], (20 * 20 * 12, 1)))
    xp = np.array([8.6, 10.0, 0.5])                  # on the first node layer: u is the node value
    xf = xp + o.trilinear(xp)
    ok, xi = o.bisect(0, xp, xf, 1)
    assert ok and o.inside(xp, 1) == -1 and o.inside(xf, 1) == 0
    assert o.reflect(0, xi, xf, 1)[2] < -0.1
    out = o.walkers_advance(xp[None, :], np.array([0], np.uint32))
    np.testing.assert_array_equal(out[0], xp)


@pytest.mark.parametrize("q", [15, 19])
def test_no_walker_ends_inside_a_moving_particle(q):
    w = I.ragged(q=q, n_walkers=3000)
    o = Oracle.from_workload(w)
    for _ in range(3):
        o.step(10)
        x, _ = o.walkers()
        inside = [o.inside(xx) for xx in x]
        assert max(inside) == -1
        assert x[:, 2].min() >= 0.0 and x[:, 2].max() <= w.dims[2]
    c = o.counters()
    assert c["type_IV"] > 0 and c["type_II"] + c["type_III"] > 0
    assert c["bisect_fail"] == 0 and c["refill_fail"] == 0 and c["wall_fail"] == 0
    assert o.concentration().sum() == w.n_walkers


def test_binning_matches_floor_and_wrap():
    o = Oracle((10, 7, 5), wall_mask=4)
    rng = np.random.default_rng(6)
    pos = np.concatenate([rng.uniform(-25, 35, (4000, 2)), rng.uniform(0, 5, (4000, 1))], 1).astype(np.float32)
    pos[:5, 2] = [0.0, 5.0, 4.9999995, 1e-7, 2.5]
    cell = o.bin_positions(pos)
    i = np.floor(pos[:, 0]).astype(np.int64) % 10
    j = np.floor(pos[:, 1]).astype(np.int64) % 7
    k = np.clip(np.floor(pos[:, 2]).astype(np.int64), 0, 4)
    assert np.array_equal(cell, (k * 7 + j) * 10 + i)


def test_moments_match_numpy():
    o = Oracle((12, 12, 12), D=0.05, seed=2)
    o.set_walkers(np.random.default_rng(7).uniform(0, 12, (5000, 3)))
    o.step(8)
    x, x0 = o.walkers()
    m = o.moments()
    assert m[0] == 5000
    assert np.allclose(m[1:4], (x - x0).mean(0), rtol=1e-12, atol=1e-15)
    assert np.allclose(m[4:7], (x - x0).var(0), rtol=1e-12)
    assert np.allclose(m[7:10], x.mean(0), rtol=1e-12)
    assert np.allclose(m[10:13], x.var(0), rtol=1e-12)


def test_seeding_is_uniform_in_the_fluid_and_exact_in_count():
    w = I.parity_single(n_walkers=20000)
    o = Oracle.from_workload(w)
    x, x0 = o.walkers()
    assert len(x) == 20000 and np.array_equal(x, x0)
    assert x.min() >= 0.0 and x.max() <= 32.0
    r = np.linalg.norm(x - 16.0, axis=1)
    assert r.min() > 6.0 - 1e-5            # none inside the k = 36 sphere (radius 6)
    # uniform over the fluid: counts in 8 octants equal (the sphere is centred)
    octant = ((x[:, 0] > 16) * 1 + (x[:, 1] > 16) * 2 + (x[:, 2] > 16) * 4)
    counts = np.bincount(octant, minlength=8)
    assert stats.chisquare(counts).pvalue > 1e-4
    # radial density outside the sphere: fraction within 6 < r < 10 matches the volume share
    shell = ((r > 6) & (r < 10)).mean()
    vol = 4 / 3 * np.pi * (1000 - 216) / (32 ** 3 - 4 / 3 * np.pi * 216)
    assert shell == pytest.approx(vol, rel=0.05)

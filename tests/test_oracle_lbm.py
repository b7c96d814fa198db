"""Pins of the oracle's lattice Boltzmann step (Eqs. 12-15) with half-way bounce-back walls,
Guo body forcing and partially-saturated solid cells."""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_2308_05007_gb300 import inputs as I


@pytest.mark.parametrize("q", [15, 19])
def test_lattice_tables(q):
    e, w = lattice(q)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose((w[:, None] * e).sum(0), 0.0, atol=1e-16)
    # second moment c_s^2 = 1/3, isotropic
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), np.eye(3) / 3, atol=1e-15)
    # fourth-order isotropy: sum w e_a^2 e_b^2 = 1/9 (a != b), sum w e_a^4 = 1/3
    m4 = np.einsum("i,ia,ib->ab", w, e ** 2, e ** 2)
    assert np.allclose(m4, np.full((3, 3), 1 / 9) + np.eye(3) * (1 / 3 - 1 / 9), atol=1e-15)
    for i in range(1, q):   # opposite pairs
        j = i + 1 if i % 2 else i - 1
        assert np.array_equal(e[i], -e[j])


@pytest.mark.parametrize("q", [15, 19])
def test_rest_state_is_a_fixed_point(q):
    o = Oracle((6, 5, 4), q=q, tau=0.7)
    f0 = o.populations()
    o.step_fluid(5)
    assert np.allclose(o.populations(), f0, rtol=0, atol=1e-15)
    assert np.abs(o.velocity()).max() < 1e-15


@pytest.mark.parametrize("q", [15, 19])
def test_uniform_flow_is_a_fixed_point(q):
    """Equilibrium at constant u in a periodic box is steady (Section 3.1's constant flow)."""
    o = Oracle((5, 4, 3), q=q, tau=0.9, init_velocity=(0.2, -0.05, 0.01))
    o.step_fluid(4)
    assert np.allclose(o.velocity(), [0.2, -0.05, 0.01], atol=1e-14)
    assert np.allclose(o.density(), 1.0, atol=1e-14)


@pytest.mark.parametrize("q", [15, 19])
def test_momentum_grows_by_body_force(q):
    """Periodic box, no solids: BGK + Guo adds exactly F per cell per step to sum_i f_i e_i."""
    F = np.array([1e-4, -3e-5, 2e-5])
    o = Oracle((7, 6, 5), q=q, tau=0.8, body_force=F)
    N = 7 * 6 * 5
    for n in (1, 2, 10):
        o.step_fluid(1 if n == 1 else n - o.t)
        mm = o.mass_momentum()
        # reported momentum is the pre-collision sum of step t = o.t - 1
        assert np.allclose(mm[1:], (o.t - 1) * F * N, rtol=1e-10, atol=1e-15)
        assert mm[0] == pytest.approx(N, rel=1e-14)


def test_oscillating_drive_adds_F0_sin_per_step():
    """The oscillator's drive F(t) = F0 sin(2 pi t / T) (Eq. 37): the momentum after the steps
    0 .. t-1 is N F0 times the sum of sin(2 pi s / T) over them."""
    F0, T = np.array([2e-4, 0.0, -1e-4]), 7.0
    o = Oracle((5, 4, 3), q=15, tau=0.9, body_force=F0, force_period=T)
    N = 5 * 4 * 3
    for n in (2, 5, 11):
        o.step_fluid(n - o.t)
        mm = o.mass_momentum()
        want = F0 * N * sum(np.sin(2 * np.pi * s / T) for s in range(o.t - 1))
        assert np.allclose(mm[1:], want, rtol=1e-10, atol=1e-16), (n, mm[1:], want)


@pytest.mark.parametrize("q,tau", [(15, 0.5 + np.sqrt(3 / 16)), (15, 0.8), (19, 1.2), (19, 0.6)])
def test_plane_poiseuille_closed_form(q, tau):
    """Force-driven flow between no-slip walls at z = 0 and z = H (half-way bounce-back).
    The steady discrete solution is the parabola F z (H - z) / (2 nu) plus a slip
    F (16 L - 3) / (24 nu), L = (tau - 1/2)^2 (He, Zou, Luo and Dembo 1997; Ginzburg and
    Adler 1994), which vanishes at tau = 1/2 + sqrt(3/16)."""
    H, F = 8, 1e-5
    nu = (tau - 0.5) / 3
    o = Oracle((1, 1, H), q=q, tau=tau, wall_mask=4, body_force=(F, 0, 0))
    o.step_fluid(int(40 * H * H / nu))
    u = o.velocity()
    z = np.arange(H) + 0.5
    lam = (tau - 0.5) ** 2
    exact = F * z * (H - z) / (2 * nu) + F * (16 * lam - 3) / (24 * nu)
    assert np.allclose(u[:, 0], exact, rtol=1e-9, atol=0)
    assert np.abs(u[:, 1:]).max() < 1e-14


def test_rectangular_duct_series_solution():
    """Force-driven flow in a square duct (walls on y and z), against the textbook Fourier
    series (e.g. White, Viscous Fluid Flow, Eq. 3-48); second-order in the grid spacing at the
    tau where half-way bounce-back is exact for the plane channel."""
    n, F = 16, 1e-6
    tau = 0.5 + np.sqrt(3 / 16)
    nu = (tau - 0.5) / 3
    o = Oracle((1, n, n), q=19, tau=tau, wall_mask=6, body_force=(F, 0, 0))
    o.step_fluid(int(12 * n * n / nu))
    u = o.velocity()[:, 0].reshape(n, n)   # [z, y]
    a = b = n / 2.0
    y = np.arange(n) + 0.5 - b
    z = np.arange(n) + 0.5 - a
    Y, Z = np.meshgrid(y, z)
    ser = np.zeros_like(Y)
    for k in range(1, 400, 2):
        ser += ((-1) ** ((k - 1) // 2) * (1 - np.cosh(k * np.pi * Y / (2 * a)) / np.cosh(k * np.pi * b / (2 * a)))
                * np.cos(k * np.pi * Z / (2 * a)) / k ** 3)
    exact = 16 * a * a * F / (nu * np.pi ** 3) * ser
    err = np.abs(u - exact).max() / exact.max()
    assert err < 5e-3, err


def _moving_particles(walls=0):
    mb = I.Metaballs(
        center_offsets=np.array([0, 2, 3], np.int32),
        centers_body=np.array([[0, 0, 0], [1.5, 0.5, 0], [0, 0, 0]], np.float32),
        k=np.array([9.0, 4.0, 12.0], np.float32),
        origin=np.array([[8.0, 8.0, 8.0], [20.0, 15.0, 9.0]]),
        amplitude=np.array([[2.0, 0.0, 1.0], [0.0, 1.5, 0.0]]),
        period=np.array([30.0, 20.0]), phase=np.array([0.0, 0.5]),
        omega=np.array([[0.0, 0.0, 0.05], [0.0, 0.0, 0.0]]))
    return mb


@pytest.mark.parametrize("q", [15, 19])
def test_mass_conservation_with_walls_and_moving_solids(q):
    o = Oracle((26, 22, 18), q=q, tau=0.75, wall_mask=4, body_force=(3e-5, 0, 0), force_period=25)
    o.set_metaballs(_moving_particles())
    N = 26 * 22 * 18
    for _ in range(4):
        o.step_fluid(5)
        assert o.mass_momentum()[0] == pytest.approx(N, rel=1e-12)


@pytest.mark.parametrize("q", [15, 19])
def test_momentum_exchange_balance(q):
    """Periodic box: the fluid momentum change over a step equals the body force on the
    fluid share minus the hydrodynamic force on the particles,
    P(t+1) - P(t) = sum_cells (1 - B) F(t) - sum_p F_p(t)."""
    tau = 0.75
    F0 = np.array([2e-5, -1e-5, 0.5e-5])
    o = Oracle((26, 22, 18), q=q, tau=tau, body_force=F0)
    o.set_metaballs(_moving_particles())
    o.step_fluid(3)
    for _ in range(6):
        t = o.t
        cnt, _ = o.solid(t)
        eps = cnt / 64.0
        B = eps * (tau - 0.5) / ((1 - eps) + (tau - 0.5))
        o.step_fluid(1)
        p_t = o.mass_momentum()[1:]
        Fp = o.forces()[:, :3].sum(0)
        o.step_fluid(1)
        p_t1 = o.mass_momentum()[1:]
        # the second step's report is the pre-collision momentum of t+1
        assert np.allclose(p_t1 - p_t, (1 - B).sum() * F0 - Fp, rtol=1e-8, atol=1e-13)
        assert np.abs(Fp).max() > 1e-8


@pytest.mark.parametrize("coupling,lo,hi", [(0, 0.80, 1.05), (1, 0.93, 1.03)])
def test_spinning_sphere_feels_the_stokes_rotational_drag(coupling, lo, hi):
    """A sphere of radius a spinning at w in still fluid feels the torque -8 pi mu a^3 w
    (Stokes flow; periodic images change it by O((a/L)^3)). The torque is exactly
    anti-parallel to w, and its size is that of the closed form to the resolution of the
    surface: partially saturated cells blur it over a cell (0.88 at a = 4); interpolated
    bounce-back places it to within a few percent."""
    n, a, tau = 24, 4.0, 1.0
    ax = np.array([1.0, -2.0, 0.5]) / np.sqrt(5.25)
    w = 0.004 * ax
    mb = I.Metaballs(center_offsets=np.array([0, 1], np.int32), centers_body=np.zeros((1, 3), np.float32),
                     k=np.array([a * a], np.float32), origin=np.array([[n / 2, n / 2, n / 2]]),
                     amplitude=np.zeros((1, 3)), period=np.zeros(1), phase=np.zeros(1), omega=np.array([w]))
    o = Oracle((n, n, n), q=19, tau=tau)
    o.set_metaballs(mb)
    o.set_coupling(coupling)
    o.step_fluid(200)
    T = o.forces()[0, 3:]
    want = -8 * np.pi * ((tau - 0.5) / 3) * a ** 3 * w
    ratio = T @ want / (want @ want)
    assert lo < ratio < hi, ratio
    assert np.linalg.norm(T - ratio * want) < 1e-3 * np.linalg.norm(want)


@pytest.mark.parametrize("centre", [(12.0, 12.0, 12.0), (0.5, 12.0, 23.5)])
def test_solid_interior_moves_with_the_particle(centre):
    """Inside a partially-saturated particle (B = 1 cells) the fluid takes the rigid-body
    velocity u_s = v + omega x r, up to the stencil-scale mixing with the fluid outside
    (under 5% three cells in from the surface). The second particle straddles two periodic
    faces: r is the minimum-image offset from its centre."""
    c = np.array(centre)
    mb = I.Metaballs(center_offsets=np.array([0, 1], np.int32),
                     centers_body=np.zeros((1, 3), np.float32), k=np.array([49.0], np.float32),
                     origin=np.array([c]), amplitude=np.array([[0.0, 0.0, 0.0]]),
                     period=np.zeros(1), phase=np.zeros(1), omega=np.array([[0.0, 0.0, 0.01]]))
    o = Oracle((24, 24, 24), q=19, tau=0.8)
    o.set_metaballs(mb)
    o.step_fluid(60)
    cnt, _ = o.solid(o.t - 1)
    u = o.velocity()
    idx = np.arange(24 ** 3)
    x = np.stack([idx % 24, idx // 24 % 24, idx // 576], 1) + 0.5
    r = x - c
    r -= 24.0 * np.round(r / 24.0)
    us = np.cross(np.array([0, 0, 0.01]), r)
    deep = (np.linalg.norm(r, axis=1) < 4.0) & (cnt == 64)
    assert deep.sum() > 100
    assert np.abs(u[deep] - us[deep]).max() < 0.05 * np.abs(us[deep]).max()
    # far outside, the fluid is nearly at rest compared with the particle surface speed
    far = np.linalg.norm(r, axis=1) > 11.0
    assert np.abs(u[far]).max() < 0.2 * 0.01 * 7.0


def test_zero_solid_fraction_is_plain_bgk():
    """A particle whose cells are all empty leaves the fluid identical to a run without it."""
    F = (1e-5, 0, 0)
    a = Oracle((12, 10, 9), q=15, tau=0.7, wall_mask=4, body_force=F)
    b = Oracle((12, 10, 9), q=15, tau=0.7, wall_mask=4, body_force=F)
    b.set_metaballs(I.single_sphere((6.0, 5.0, 4.5), 1e-3))   # radius 0.03: no sub-sample hit
    assert b.solid(0)[0].sum() == 0
    a.step_fluid(7)
    b.step_fluid(7)
    assert np.array_equal(a.populations(), b.populations())

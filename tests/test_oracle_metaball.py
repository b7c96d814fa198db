"""Pins of the oracle's particle geometry: Eq. 3 (metaball), Eq. 17 (gradient), the prescribed
rigid motion, the bound radius, and the sub-sampled solid fraction."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2308_05007_gb300 import inputs as I


def _two_ball():
    mb = I.Metaballs(
        center_offsets=np.array([0, 3, 4], np.int32),
        centers_body=np.array([[0, 0, 0], [2.5, 0.5, 0], [-1, 2, 1], [0, 0, 0]], np.float32),
        k=np.array([9.0, 6.0, 4.0, 16.0], np.float32),
        origin=np.array([[10.0, 9.0, 8.5], [3.0, 4.0, 12.0]]),
        amplitude=np.array([[1.5, 0, 0.5], [0, 2.0, 0]]),
        period=np.array([50.0, 30.0]), phase=np.array([0.2, 1.0]),
        omega=np.array([[0, 0, 0.03], [0.01, 0.02, 0]]))
    return mb


def test_single_centre_value_and_surface_radius():
    o = Oracle((32, 32, 32))
    o.set_metaballs(I.single_sphere((16.0, 16.0, 16.0), 36.0))
    for r in (1.0, 3.0, 6.0, 9.5):
        f, g = o.metaball(0, [16.0 + r, 16.0, 16.0])
        assert f == pytest.approx(36.0 / r ** 2, rel=1e-14)
        # Eq. 17 radial component: -2 k r / r^4
        assert g[0] == pytest.approx(-2 * 36.0 / r ** 3, rel=1e-14)
    # surface f = 1 at r = sqrt(k); the bound radius is exact for one centre
    assert o.bound_radius(0) == pytest.approx(6.0, abs=1e-9)
    assert o.inside([16 + 5.999, 16, 16]) == 0
    assert o.inside([16 + 6.001, 16, 16]) == -1


def test_gradient_matches_finite_differences():
    o = Oracle((24, 24, 24))
    o.set_metaballs(_two_ball())
    rng = np.random.default_rng(0)
    for t in (0, 7, 19):
        for _ in range(20):
            x = rng.uniform(0, 24, 3)
            p = int(rng.integers(0, 2))
            f, g = o.metaball(p, x, t)
            h = 1e-5
            fd = np.array([(o.metaball(p, x + h * e, t)[0] - o.metaball(p, x - h * e, t)[0]) / (2 * h)
                           for e in np.eye(3)])
            assert np.allclose(g, fd, rtol=1e-5, atol=1e-7 * max(1.0, abs(f)))


def test_binary32_metaball_close_to_fp64():
    o = Oracle((24, 24, 24))
    o.set_metaballs(_two_ball())
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = rng.uniform(0, 24, 3).astype(np.float32)
        f64, _ = o.metaball(1, x.astype(np.float64), 3)
        f32 = o.metaball32(1, x, 3)
        assert abs(float(f32) - f64) <= 2e-6 * f64 + 1e-12


def test_prescribed_pose_and_velocity():
    o = Oracle((24, 24, 24))
    mb = _two_ball()
    o.set_metaballs(mb)
    for p in range(2):
        for t in (0, 5, 33):
            org, vel = o.pose(p, t)
            th = 2 * np.pi * t / mb.period[p] + mb.phase[p]
            assert np.allclose(org, mb.origin[p] + mb.amplitude[p] * np.sin(th), atol=1e-13)
            # velocity is the time derivative of the origin (central difference in t)
            h = 1e-4
            op = mb.origin[p] + mb.amplitude[p] * np.sin(2 * np.pi * (t + h) / mb.period[p] + mb.phase[p])
            om = mb.origin[p] + mb.amplitude[p] * np.sin(2 * np.pi * (t - h) / mb.period[p] + mb.phase[p])
            assert np.allclose(vel, (op - om) / (2 * h), atol=1e-7)


def test_rotation_moves_control_points_rigidly():
    """A single off-centre control point spinning about z: f = k / r^2 about the rotated point."""
    mb = I.Metaballs(center_offsets=np.array([0, 1], np.int32),
                     centers_body=np.array([[3.0, 0.0, 0.0]], np.float32),
                     k=np.array([4.0], np.float32), origin=np.array([[12.0, 12.0, 12.0]]),
                     amplitude=np.zeros((1, 3)), period=np.zeros(1), phase=np.zeros(1),
                     omega=np.array([[0.0, 0.0, 0.1]]))
    o = Oracle((24, 24, 24))
    o.set_metaballs(mb)
    for t in (0, 4, 11):
        a = 0.1 * t
        c = np.array([12 + 3 * np.cos(a), 12 + 3 * np.sin(a), 12.0])
        x = c + np.array([0.5, -0.25, 1.0])
        f, _ = o.metaball(0, x, t)
        assert f == pytest.approx(4.0 / (0.25 + 0.0625 + 1.0), rel=1e-12)


def test_periodic_minimum_image():
    """A particle at the box edge acts through the periodic face."""
    o = Oracle((20, 20, 20))
    o.set_metaballs(I.single_sphere((0.5, 10.0, 10.0), 9.0))
    f, _ = o.metaball(0, [19.5, 10.0, 10.0])
    assert f == pytest.approx(9.0, rel=1e-14)
    assert o.inside([18.0, 10.0, 10.0]) == 0


def test_bound_radius_is_a_bound():
    """No point farther than the bound radius from the origin reaches f = 1 (random rays)."""
    rng = np.random.default_rng(3)
    w = I.ragged()
    o = Oracle(w.dims, wall_mask=w.wall_mask)
    o.set_metaballs(w.metaballs)
    mb = w.metaballs
    for p in range(mb.n_particles):
        R = o.bound_radius(p)
        cb = mb.centers_body[mb.center_offsets[p]:mb.center_offsets[p + 1]].astype(np.float64)
        kk = mb.k[mb.center_offsets[p]:mb.center_offsets[p + 1]].astype(np.float64)
        assert R >= np.max(np.linalg.norm(cb, axis=1))
        dirs = rng.normal(size=(500, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        pts = dirs * (R + 1e-6)
        f = (kk[None, :] / ((pts[:, None, :] - cb[None]) ** 2).sum(-1)).sum(-1)
        assert f.max() < 1.0


def _brute_solid(dims, walls, mb, t):
    """Every sub-sample of every cell against every particle, in numpy binary32 with the same
    operation order as the oracle's decision (no bound radius skipping)."""
    o = Oracle(dims, wall_mask=walls)
    o.set_metaballs(mb)
    n = np.array(dims, np.float32)
    # world control points at t come from the oracle's FP64 pose, rounded to binary32
    cw = []
    for p in range(mb.n_particles):
        org, _ = o.pose(p, t)
        cb = mb.centers_body[mb.center_offsets[p]:mb.center_offsets[p + 1]].astype(np.float64)
        w = mb.omega[p]
        wn = np.linalg.norm(w)
        R = np.eye(3)
        if wn > 0:
            ax = w / wn
            K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
            ang = wn * t
            R = np.cos(ang) * np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * np.outer(ax, ax)
        c = org[None, :] + cb @ R.T
        for a in range(3):
            if not (walls >> a & 1):
                c[:, a] -= dims[a] * np.floor(c[:, a] / dims[a])
        cw.append(c.astype(np.float32))
    nx, ny, nz = dims
    off = (np.float32(0.125) + np.float32(0.25) * np.arange(4, dtype=np.float32))
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ii, jj, kk], -1).astype(np.float32)   # [nx, ny, nz, 3]
    sub = np.stack(np.meshgrid(off, off, off, indexing="ij"), -1).reshape(64, 3)  # (cx, cy, cz)
    xs = base[..., None, :] + sub[None, None, None, :, :]   # [nx, ny, nz, 64, 3]
    inside = np.zeros((mb.n_particles,) + xs.shape[:-1], bool)
    for p in range(mb.n_particles):
        kp = mb.k[mb.center_offsets[p]:mb.center_offsets[p + 1]].astype(np.float32)
        f = np.zeros(xs.shape[:-1], np.float32)
        for i in range(len(kp)):
            d = []
            for a in range(3):
                da = xs[..., a] - cw[p][i, a]
                if not (walls >> a & 1):
                    h = np.float32(0.5) * n[a]
                    da = np.where(da > h, da - n[a], np.where(da < -h, da + n[a], da)).astype(np.float32)
                d.append(da)
            r2 = (d[0] * d[0] + d[1] * d[1]).astype(np.float32)
            r2 = (r2 + d[2] * d[2]).astype(np.float32)
            with np.errstate(divide="ignore"):
                f = (f + kp[i] / r2).astype(np.float32)
        inside[p] = f >= np.float32(1.0)
    count = inside.any(0).sum(-1)                        # [nx, ny, nz]
    per = inside.sum(-1)                                  # [P, nx, ny, nz]
    owner = np.where(count > 0, np.argmax(per, axis=0), -1)
    # oracle layout: x fastest
    return count.transpose(2, 1, 0).ravel(), owner.transpose(2, 1, 0).ravel(), o


@pytest.mark.parametrize("t", [0, 9])
def test_solid_fraction_equals_brute_force(t):
    dims, walls = (16, 14, 13), 4
    mb = _two_ball()
    mb.origin[:, 2] = [6.5, 6.0]
    cnt_b, own_b, o = _brute_solid(dims, walls, mb, t)
    cnt, own = o.solid(t)
    assert np.array_equal(cnt, cnt_b)
    assert np.array_equal(own, own_b)
    assert cnt.max() == 64 and (cnt > 0).sum() > 50


@pytest.mark.parametrize("t", [0, 9])
def test_sampled_solid_fraction_equals_brute_force(t):
    """The cell-list entry (used to time bounded samples) gives the brute-force counts and
    owners of exactly the listed cells, in list order, repeats included."""
    dims, walls = (16, 14, 13), 4
    mb = _two_ball()
    mb.origin[:, 2] = [6.5, 6.0]
    cnt_b, own_b, o = _brute_solid(dims, walls, mb, t)
    cells = np.random.default_rng(5).integers(0, cnt_b.size, 700)
    cells[:3] = [0, cnt_b.size - 1, 0]
    cnt, own = o.solid_cells(cells, t)
    assert np.array_equal(cnt, cnt_b[cells])
    assert np.array_equal(own, own_b[cells])
    assert (cnt > 0).any() and (cnt == 0).any()


def test_owner_ties_go_to_the_lower_index():
    """Two equal spheres mirror-symmetric about the centre plane of cell (8, 8, 8) hold equal
    sub-sample counts there (all 64 each, evaluated exactly alike in binary32). The tie gives the
    cell to the lower particle index, and the brute force agrees on every cell."""
    mb = I.Metaballs(center_offsets=np.array([0, 1, 2], np.int32), centers_body=np.zeros((2, 3), np.float32),
                     k=np.array([6.25, 6.25], np.float32),
                     origin=np.array([[6.5, 8.5, 8.5], [10.5, 8.5, 8.5]]), amplitude=np.zeros((2, 3)),
                     period=np.zeros(2), phase=np.zeros(2), omega=np.zeros((2, 3)))
    dims = (17, 17, 17)
    cnt_b, own_b, o = _brute_solid(dims, 0, mb, 0)
    cnt, own = o.solid(0)
    c = 8 + 17 * (8 + 17 * 8)
    assert cnt[c] == 64 and own[c] == 0
    assert np.array_equal(cnt, cnt_b) and np.array_equal(own, own_b)
    assert (own == 1).any()


def test_solid_fraction_sphere_volume():
    """Sum of epsilon over cells converges to the sphere volume (4/3) pi r^3."""
    for r, c in ((6.0, (16.0, 16.0, 16.0)), (4.5, (10.3, 11.7, 9.1))):
        o = Oracle((32, 32, 32))
        o.set_metaballs(I.single_sphere(c, r * r))
        cnt, _ = o.solid(0)
        vol = cnt.sum() / 64.0
        assert vol == pytest.approx(4 / 3 * np.pi * r ** 3, rel=0.01)
        # every cell wholly inside the sphere is fully solid, every cell wholly outside empty
        idx = np.arange(32 ** 3)
        cx = np.stack([idx % 32, idx // 32 % 32, idx // 1024], 1) + 0.5
        dist = np.linalg.norm(cx - np.array(c), axis=1)
        assert np.all(cnt[dist < r - 0.87] == 64)
        assert np.all(cnt[dist > r + 0.87] == 0)

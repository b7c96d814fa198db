"""Free DEM on the GPU (Section 2.2, Eqs. 4-11) against the FP64 CPU oracle.

- Fluid force off (hydro = 0): the particle trajectories do not depend on the fluid, and the
  DEM kernels round every binary64 operation as the oracle does (no contraction, IEEE division
  and square root, the same operation order), so the states agree bit for bit through contacts
  between particles and with the walls.
- Fluid force on: one step from the GPU's own state (populations, velocity, particles) against
  the oracle. The particles' new velocities differ only through the hydrodynamic force, which
  the GPU forms in binary32 (relative 1e-4 of the force, times dt / m).
- The three schedules, graph replay and a checkpoint restart give identical results.
- With the paper's IBB coupling: one coupled step against the oracle (given the previous step's
  node classes), and identical schedules and graphs.
- Set-ups the library cannot run (binary16 or unshifted binary32 storage) are refused.
"""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2308_05007_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300 import rwmi
    rwmi.load()
    yield


def _converging(hydro=0, seed=11, n_particles=4, speed=0.1):
    """dem_box with every particle aimed at the common centre, so that contacts follow."""
    w = I.dem_box(n_particles=n_particles, seed=seed, hydro=hydro)
    o = w.metaballs.origin
    aim = o.mean(0) - o
    w.dem.velocity[:] = speed * aim / np.linalg.norm(aim, axis=1, keepdims=True)
    return w


def test_mass_properties_bit_exact():
    """Mass, centre of mass and inertia from the metaball sample sums: integers on both sides, the
    same binary32 inside test and the same binary64 formulas, so they agree bit for bit; the
    recentred control points give the same solid fraction at the start."""
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.oscillator_dem(n=96, n_particles=3, n_walkers=0)
    ora = Oracle.from_workload(w, seed_walkers=False)
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        np.testing.assert_array_equal(sim.particle_mass(), ora.dem_mass())
        np.testing.assert_array_equal(sim.particle_state(), ora.particle_state())
        cg, og = sim.solid()
    co, oo = ora.solid(ora.t)
    assert np.array_equal(cg, co) and np.array_equal(og, oo)


def test_trajectories_bit_exact_without_fluid_force():
    from paper_2308_05007_gb300.rwmi import Simulation
    w = _converging(hydro=0)
    ora = Oracle.from_workload(w, seed_walkers=False)
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        g0 = sim.particle_state()
        np.testing.assert_array_equal(g0, ora.particle_state())
        touched = False
        for chunk in range(8):
            sim.step(20)
            ora.dem_advance(20)
            st = sim.particle_state()
            np.testing.assert_array_equal(st, ora.particle_state(), err_msg=f"after {20 * (chunk + 1)} steps")
            free = g0[:, 7:10] + (20 * (chunk + 1)) * np.asarray(w.dem.gravity)
            touched |= bool(np.abs(st[:, 7:10] - free).max() > 1e-6)
    assert touched, "no contact happened"


def test_many_particles_take_the_two_launch_path_bit_exactly():
    """More than 128 particles: two launches per DEM step instead of one block; the same slot and
    integration code, so still bit-identical to the oracle (fluid force off), contacts included."""
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.dem_box(dims=(96, 96, 96), n_particles=130, seed=21, hydro=0, n_walkers=0, speed=0.12)
    o = w.metaballs.origin
    aim = o.mean(0) - o
    w.dem.velocity[:] = 0.12 * aim / np.linalg.norm(aim, axis=1, keepdims=True)
    ora = Oracle.from_workload(w, seed_walkers=False)
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        g0 = sim.particle_state()
        np.testing.assert_array_equal(g0, ora.particle_state())
        sim.step(140)
        ora.dem_advance(140)
        st = sim.particle_state()
    np.testing.assert_array_equal(st, ora.particle_state())
    free = g0[:, 7:10] + 140 * np.asarray(w.dem.gravity)
    assert (np.abs(st[:, 7:10] - free).max(1) > 1e-6).sum() > 10, "too few contacts"


def test_solid_fraction_follows_the_dem_state():
    """The raster of a free-DEM run uses the particle state: bit-exact against the oracle's
    rasteriser fed the same state."""
    from paper_2308_05007_gb300.rwmi import Simulation
    w = _converging(hydro=0)
    ora = Oracle.from_workload(w, seed_walkers=False)
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        sim.step(37)
        st = sim.particle_state()
        cg, og = sim.solid()
    ora.set_particle_state(st)
    co, oo = ora.solid(ora.t)
    assert np.array_equal(cg, co) and np.array_equal(og, oo)
    assert (cg > 0).sum() > 100


def test_coupled_step_from_identical_state():
    from paper_2308_05007_gb300.rwmi import Simulation
    from oracle.oracle import lattice
    w = I.dem_box(n_particles=3, seed=4, speed=0.0, gravity=(0.0, 0.0, -2e-4), hydro=1, n_walkers=0)
    w = I.with_(w, body_force=(3e-5, 0.0, 0.0))
    w.dem.velocity[:] = 0.0
    w.dem.spin[:] = 0.0
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        eg, _ = sim.lattice()
        eo, _ = lattice(w.q)
        perm = np.array([int(np.where((eg == eo[i]).all(1))[0][0]) for i in range(w.q)])
        sim.step(12)
        t = sim.t
        f0 = sim.populations()[perm]
        st0 = sim.particle_state()
        sim.step(1)
        st1 = sim.particle_state()
        Fg = sim.particle_forces()
        mp = sim.particle_mass()
    ora = Oracle.from_workload(w, seed_walkers=False)
    ora.set_populations(f0)
    ora.set_time(t)
    ora.set_particle_state(st0)
    ora.step_fluid(1)
    Fo = ora.forces()
    so = ora.particle_state()
    assert np.abs(Fo[:, :3]).max() > 1e-4   # the fluid does push
    tolF = 2e-4 * np.abs(Fo[:, :3]).max()
    # the torque is a sum of r x F terms over the particle's cells that largely cancel: its error
    # is the force error times the lever arm (the particle's radius plus two cells)
    radius = (3.0 * mp[:, 0].max() / (4.0 * np.pi * w.dem.density)) ** (1.0 / 3.0) + 2.0
    tolT = tolF * radius
    np.testing.assert_allclose(Fg[:, :3], Fo[:, :3], rtol=0, atol=tolF)
    np.testing.assert_allclose(Fg[:, 3:], Fo[:, 3:], rtol=0, atol=tolT)
    # one LBM step = the DEM steps of dt = 1 / substeps: velocity error <= force error / m, origin
    # error <= that (times sum of dt k dt <= 1), spin error <= torque error / smallest inertia
    dv = tolF / mp[:, 0].min()
    dw = tolT / mp[:, 4:7].min()
    assert np.abs(st1[:, 7:10] - so[:, 7:10]).max() <= dv + 1e-15
    assert np.abs(st1[:, :3] - so[:, :3]).max() <= dv + 1e-12
    assert np.abs(st1[:, 10:13] - so[:, 10:13]).max() <= dw + 1e-15
    assert np.abs(st1[:, 7:10] - st0[:, 7:10]).max() > 100 * dv   # the step moved them


def test_schedules_graphs_and_restart_agree(tmp_path):
    from paper_2308_05007_gb300.rwmi import Simulation
    w = _converging(hydro=1)
    ref = None
    for overlap in (0, 1, 2):
        for graphs in (False, True):
            with Simulation.from_workload(w, overlap=overlap, use_graphs=graphs, sort_interval=4) as s:
                s.step(30)
                pos, _ = s.walkers_by_id()
                res = (s.particle_state(), s.populations(), pos)
            if ref is None:
                ref = res
            else:
                for a, b in zip(ref, res):
                    assert np.array_equal(a, b), (overlap, graphs)
    path = os.fspath(tmp_path / "dem.ckpt")
    with Simulation.from_workload(w, sort_interval=4) as s:
        s.step(14)
        s.save(path)
        s.step(16)
        want = (s.particle_state(), s.populations())
    with Simulation.from_workload(w, sort_interval=4) as s:
        s.load(path)
        s.step(16)
        got = (s.particle_state(), s.populations())
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    # a free-DEM checkpoint does not load into a context with prescribed motion
    from paper_2308_05007_gb300.rwmi import RwmiError
    with Simulation.from_workload(I.with_(w, dem=None), sort_interval=4) as s:
        with pytest.raises(RwmiError):
            s.load(path)


def test_refused_setups():
    from paper_2308_05007_gb300.rwmi import RwmiError, Simulation
    for kw in (dict(storage=2), dict(storage=0)):
        w = I.with_(_converging(), **kw)
        with pytest.raises(RwmiError):
            Simulation.from_workload(w, seed_walkers=False)


@pytest.mark.parametrize("storage", [1, 3])
def test_ibb_coupled_step_from_identical_state(storage):
    """The paper's own pairing: free particles with interpolated bounce-back, momentum exchange
    and refilling (Section 2.4.3). One step from the GPU's state against the oracle, which is
    given the same populations, velocity (u_f, u_ff of Eq. 24), particle state and node classes
    of the previous step; the forces and the new particle state agree within the LBM update's
    precision (binary64 storage: 1e-9 of the force)."""
    from paper_2308_05007_gb300.rwmi import Simulation
    from oracle.oracle import lattice
    w = I.dem_box(n_particles=3, seed=4, speed=0.0, gravity=(0.0, 0.0, -2e-4), hydro=1, n_walkers=0,
                  storage=storage)
    w = I.with_(w, body_force=(3e-5, 0.0, 0.0), coupling=1)
    w.dem.velocity[:] = 0.0
    w.dem.spin[:] = 0.0
    with Simulation.from_workload(w, seed_walkers=False) as sim:
        eg, _ = sim.lattice()
        eo, _ = lattice(w.q)
        perm = np.array([int(np.where((eg == eo[i]).all(1))[0][0]) for i in range(w.q)])
        sim.step(11)
        nodes_prev = sim.nodes()
        sim.step(1)
        t = sim.t
        f0 = sim.populations()[perm]
        u0 = sim.velocity().astype(np.float64)
        st0 = sim.particle_state()
        sim.step(1)
        st1 = sim.particle_state()
        Fg = sim.particle_forces()
        mp = sim.particle_mass()
    ora = Oracle.from_workload(w, seed_walkers=False)
    ora.set_populations(f0)
    ora.set_velocity(u0)
    ora.set_time(t)
    ora.set_particle_state(st0)
    ora.set_prev_nodes(t - 1, nodes_prev)
    ora.step_fluid(1)
    Fo = ora.forces()
    so = ora.particle_state()
    assert np.abs(Fo[:, :3]).max() > 1e-4
    rel = 1e-9 if storage == 3 else 2e-4
    tolF = rel * np.abs(Fo[:, :3]).max()
    radius = (3.0 * mp[:, 0].max() / (4.0 * np.pi * w.dem.density)) ** (1.0 / 3.0) + 2.0
    tolT = tolF * radius
    np.testing.assert_allclose(Fg[:, :3], Fo[:, :3], rtol=0, atol=tolF)
    np.testing.assert_allclose(Fg[:, 3:], Fo[:, 3:], rtol=0, atol=tolT)
    dv = tolF / mp[:, 0].min()
    dw = tolT / mp[:, 4:7].min()
    assert np.abs(st1[:, 7:10] - so[:, 7:10]).max() <= dv + 1e-15
    assert np.abs(st1[:, :3] - so[:, :3]).max() <= dv + 1e-12
    assert np.abs(st1[:, 10:13] - so[:, 10:13]).max() <= dw + 1e-15


def test_ibb_schedules_and_graphs_agree():
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.with_(_converging(hydro=1), coupling=1)
    ref = None
    for overlap in (0, 2):
        for graphs in (False, True):
            with Simulation.from_workload(w, overlap=overlap, use_graphs=graphs, sort_interval=4) as s:
                s.step(20)
                res = (s.particle_state(), s.populations())
            if ref is None:
                ref = res
            else:
                for a, b in zip(ref, res):
                    assert np.array_equal(a, b), (overlap, graphs)

"""The TMA-staged LBM update (rows of 128 cells copied into shared memory by tensor copies)
against the direct-load update and against the FP64 oracle.

Both updates run the same per-cell arithmetic on the same pulled values, so every population,
velocity and walker must agree bit for bit (forces and sums up to the order of their FP64
atomics); the cases cover one partial tile per row
(nx < 128), two tiles with a partial second one (nx = 132, 136), whole tiles (nx = 256), binary32
shifted and unshifted and binary16 storage, D3Q15 and D3Q19, periodic x with its wrapped halo,
and walls on every axis (bounce-back rows read from global memory).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_2308_05007_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300 import rwmi
    rwmi.load()   # raises if the library is missing: no fallback
    yield


def _sims(w):
    from paper_2308_05007_gb300.rwmi import Simulation
    return (Simulation.from_workload(w, seed_walkers=True, lbm_staging=1),
            Simulation.from_workload(w, seed_walkers=True, lbm_staging=0))


@pytest.mark.parametrize("q,storage,walls,dims", [
    (15, 1, 4, (256, 24, 20)),
    (19, 1, 0, (132, 20, 18)),
    (15, 2, 0, (64, 30, 22)),
    (19, 0, 3, (136, 24, 22)),
    (15, 1, 7, (40, 36, 26)),
    (19, 2, 4, (136, 22, 21)),
])
def test_staged_update_is_bit_identical_to_direct_loads(q, storage, walls, dims):
    w = I.ragged(dims=dims, q=q, storage=storage, walls=walls, seed=5 + q + walls, n_walkers=2000)
    staged, direct = _sims(w)
    for n in (1, 6, 25):   # eager and captured runs, reduction steps among them
        staged.step(n)
        direct.step(n)
        assert np.array_equal(staged.populations(), direct.populations())
        assert np.array_equal(staged.velocity(), direct.velocity())
        # FP64 sums through atomics: their order may differ between runs
        assert np.allclose(staged.particle_forces(), direct.particle_forces(), rtol=1e-12, atol=1e-15)
        assert np.allclose(staged.mass_momentum(), direct.mass_momentum(), rtol=1e-12, atol=1e-15)
    for a, b in zip(staged.walkers(), direct.walkers()):
        assert np.array_equal(a, b)
    assert staged.sync() == 0 and direct.sync() == 0
    staged.close()
    direct.close()


@pytest.mark.parametrize("q,walls,dims", [(15, 4, (132, 20, 16)), (19, 0, (260, 12, 12))])
def test_staged_one_step_against_the_oracle(q, walls, dims):
    """Rows of two and three tiles (the last one partial) against the FP64 oracle, with the
    one-step tolerances of the direct update (1e-6 of max|f|, 1e-6 of max(max|u|, 0.01))."""
    w = I.ragged(dims=dims, q=q, storage=1, walls=walls, seed=21 + q, n_walkers=0)
    from paper_2308_05007_gb300.rwmi import Simulation
    sim = Simulation.from_workload(w, seed_walkers=False, lbm_staging=1)
    ora = Oracle.from_workload(w, seed_walkers=False)
    eg, wg = sim.lattice()
    eo, wo = lattice(q)
    perm = np.array([int(np.where((eg == eo[i]).all(1))[0][0]) for i in range(q)])
    sim.step(5)
    f_prev = sim.populations()[perm]
    t = sim.t
    sim.step(1)
    f_next = sim.populations()[perm]
    u_g = sim.velocity()
    ora.set_populations(f_prev)
    ora.set_time(t)
    fo, uo, _ = ora.lbm_cells(np.arange(ora.n_cells))
    assert np.abs(f_next - fo).max() <= 1e-6 * np.abs(fo).max()
    assert np.abs(u_g - uo).max() <= 1e-6 * max(np.abs(uo).max(), 1e-2)
    sim.close()


def test_a_tma_wait_that_expires_is_reported_and_the_context_stays_usable():
    """rwmi_inject_wait_timeout leaves one tile's copies unissued (its mbarrier never completes,
    nothing faults): the owning block gives up after its short bound, rwmi_sync reports
    RWMI_E_TIMEOUT, and the next steps run normally."""
    import time
    from paper_2308_05007_gb300 import rwmi
    w = I.ragged(dims=(256, 24, 20), q=15, storage=1, walls=4, seed=31, n_walkers=1000)
    sim = rwmi.Simulation.from_workload(w, seed_walkers=True, lbm_staging=1, use_graphs=False)
    sim.step(2)
    assert sim.sync() == 0
    assert rwmi.inject_wait_timeout(1) == 0
    t0 = time.perf_counter()
    sim.step(1)
    with pytest.raises(rwmi.RwmiError) as e:
        sim.sync()
    assert e.value.status == -5, str(e.value)
    assert time.perf_counter() - t0 < 5.0
    assert rwmi.inject_wait_timeout(0) == 0   # the one injected launch was taken
    sim.step(3)
    assert sim.sync() == 0
    sim.close()

"""The per-step force series (rwmi_config.force_interval, rwmi_force_series) on the GPU.

- Every row equals the forces the FP64 oracle gives after the same number of fluid steps, to the
  tolerance of the single-read force check (5e-5 of the largest component: the binary32
  velocity error carried into -B sum Omega e), for PSM with moving, spinning particles between
  walls.
- Rows recorded every 3 steps in captured graphs equal the rows of every third step recorded
  eagerly step by step: a recorded step runs the fused update-and-reduce pass, whose update stores
  the same bits as the plain update, so the trajectory and the force of each step are the same
  whatever the cadence.
- That bit-identity, for every instantiation that takes the fused pass (D3Q15/D3Q19,
  binary32-shifted and binary64 storage, walls or periodic, partially saturated cells or IBB):
  a run reduced on every step equals a run reduced on its last step only.
- The last row equals rwmi_particle_forces read after the same step.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2308_05007_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300 import rwmi
    rwmi.load()
    yield


def test_force_series_follows_the_oracle_step_by_step():
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.ragged(q=15, storage=1, walls=4, seed=17, n_walkers=0)
    sim = Simulation.from_workload(w, seed_walkers=False, force_interval=1)
    ora = Oracle.from_workload(w, seed_walkers=False)
    sim.step(8)
    steps, F = sim.force_series()
    assert list(steps) == list(range(1, 9))
    for k in range(8):
        ora.step_fluid(1)
        fo = ora.forces()
        scale = np.abs(fo[:, :3]).max()
        assert scale > 0
        assert np.abs(F[k][:, :3] - fo[:, :3]).max() <= 5e-5 * scale, k
    assert np.array_equal(F[-1], sim.particle_forces())
    sim.close()


def test_force_series_cadence_and_graphs_do_not_change_the_rows():
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.ragged(q=19, storage=1, walls=4, seed=23, n_walkers=2000)
    every = Simulation.from_workload(w, force_interval=1, use_graphs=False)
    third = Simulation.from_workload(w, force_interval=3, use_graphs=True)
    for _ in range(12):
        every.step(1)
    third.step(12)
    s1, F1 = every.force_series()
    s3, F3 = third.force_series()
    assert list(s3) == [3, 6, 9, 12]
    np.testing.assert_allclose(F3, F1[2::3], rtol=1e-12, atol=1e-12 * np.abs(F1).max())
    assert np.array_equal(every.populations(), third.populations())
    every.close()
    third.close()


@pytest.mark.parametrize("q,storage,walls,coupling", [
    (15, 1, 4, 0), (15, 1, 0, 0), (19, 1, 4, 0), (19, 1, 0, 0),
    (15, 3, 4, 0), (19, 3, 0, 0), (15, 1, 4, 1), (19, 3, 4, 1)])
def test_fused_reduction_pass_updates_bit_identically(q, storage, walls, coupling):
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.with_(I.ragged(q=q, storage=storage, walls=walls, seed=29, n_walkers=0), coupling=coupling)
    every = Simulation.from_workload(w, seed_walkers=False, force_interval=1, use_graphs=False)
    last = Simulation.from_workload(w, seed_walkers=False, use_graphs=False)
    every.step(6)   # every step reduced: the fused pass six times
    last.step(6)    # one eager call: only its last step reduced
    assert np.array_equal(every.populations(), last.populations())
    assert np.array_equal(every.velocity(), last.velocity())
    np.testing.assert_allclose(every.force_series()[1][-1], last.particle_forces(), rtol=1e-12,
                               atol=1e-12 * max(np.abs(last.particle_forces()).max(), 1e-300))
    every.close()
    last.close()

"""Failure detection of the bounded device waits, without a GPU fault: with
the wait limit set to one polling iteration, the grid barrier of the
cooperative sub-step kernel (7 CTAs here, K of about 25 with two barriers per
sub-step) and the look-back of the cell-list scan give up, the step reports
SPHFSI_E_TIMEOUT at the sync, later steps are refused, and after a checkpoint
is restored (default limit) the context steps on bit for bit like one that
never timed out.  Every wait in these kernels is bounded and every kernel
that reads cell ranges returns once the scan has given up, so nothing hangs
and nothing reads outside its arrays."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import SphError, Simulation  # noqa: E402

E_TIMEOUT = -6


def _sim(case, K):
    sim = Simulation.from_case(case)
    sim.set_solid_path(2)          # the cooperative grid kernel and its grid barrier
    sim.set_substeps(K)
    return sim


def test_a_wait_that_gives_up_is_reported_and_a_checkpoint_recovers():
    case = fc.dam_gate(seed=0)
    ref = O.OracleSim(case)
    dt, _, dts = ref.suggest_dt(vmax_f=0.0)
    K = ref.substeps(dt, dts)
    assert K > 10
    sim = _sim(case, K)
    for _ in range(2):
        sim.step(dt)
    sim.sync()
    blob = sim.get_state()
    sim.set_wait_limit(1)
    sim.step(dt)
    with pytest.raises(SphError) as e:
        sim.sync()
    assert e.value.code == E_TIMEOUT
    assert sim.info()["status"] & 2
    with pytest.raises(SphError) as e:       # refused until a checkpoint is restored
        sim.step(dt)
    assert e.value.code == E_TIMEOUT
    sim.set_wait_limit(0)
    sim.set_state(blob)
    for _ in range(3):
        sim.step(dt)
    sim.sync()
    other = _sim(case, K)
    for _ in range(5):
        other.step(dt)
    other.sync()
    for a, b in ((sim.get_fluid(), other.get_fluid()), (sim.get_solid(), other.get_solid())):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert sim.info()["step"] == other.info()["step"] == 5
    sim.close()
    other.close()

"""Flow-induced vibration channel (Section 4.1; the flag behind the cylinder
at dp_F = D/10, dp_S = D/20: 10.1k fluid, 596 solid particles) started
impulsively (reading R20): the flag-tip displacement after 1000 coarse steps
matches the FP64 oracle within 1e-3, relative to max(|u|, 0.01 dp_S), the
workload's tolerance for the tip."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import Simulation  # noqa: E402


def test_flag_tip_parity_1000_steps():
    case = fc.channel_flag(seed=0)
    assert case.inflow_tramp == 0.0     # impulsive start
    ref = O.OracleSim(case, threaded=True)
    dt, _, dts = ref.suggest_dt()
    K = ref.substeps(dt, dts)
    sim = Simulation.from_case(case)
    sim.set_substeps(K)
    sim.run(1000, dt)
    sim.sync()
    for _ in range(1000):
        ref.step(dt, K)
    s = sim.get_solid()
    tip = case.tip
    u_g = s["r"][tip] - case.s_r0[tip]
    u_o = ref.s_r[tip] - case.s_r0[tip]
    err = np.linalg.norm(u_g - u_o) / max(np.linalg.norm(u_o), 0.01 * case.s_dp)
    print("K", K, "dt", dt, "tip u oracle", u_o, "gpu", u_g, "rel err", err)
    assert np.linalg.norm(u_o) > 0.1 * case.s_dp   # the flag moved
    assert err < 1e-3
    sim.close()

"""Pulsatile flow through the venous valve (Section 4.3) through the C-ABI
on the GPU, against the oracle: the Womersley inflow profile (Appendix A)
imposed in the buffer, the two clamped leaflets with K of order 40 solid
sub-steps, one coarse step at a time."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import Simulation, SphError  # noqa: E402

ACC_TOL = 1e-5


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("wo", [1.0, 10.0])
def test_valve_steps_match_oracle(wo):
    case = fc.venous_valve(seed=2, wo=wo, DH=2e-3, L_H=4.0)
    ref = O.OracleSim(case)
    sim = Simulation.from_case(case)
    for n in range(3):
        sim.step(0.0)
        sim.sync()
        info = sim.info()
        if n == 0:
            dt, _, dts = ref.suggest_dt()
            assert abs(info["last_dt"] - dt) <= 1e-6 * dt
            assert info["last_K"] == ref.substeps(info["last_dt"], dts) and info["last_K"] > 10
        # particles in the inflow buffer at the step's start take the Womersley
        # velocity of that time before the kick
        inb = ref.f_r[:, 0] < case.inflow_width
        ref.step(info["last_dt"], info["last_K"])
        g = sim.get_fluid()
        e = {"dvdt": rel(g["dvdt"], ref.f_dvdt), "drho": rel(g["drho"], ref.f_drho), "v": rel(g["v"], ref.f_v),
             "v_buffer": rel(g["v"][inb], ref.f_v[inb])}
        s = sim.get_solid()
        e["fF"] = rel(s["fF"], ref.s_fF)
        e["F-I"] = rel(s["F"] - np.eye(2), ref.s_F - np.eye(2))
        e["abar"] = rel(s["abar"], ref.s_abar)
        assert np.abs(g["r"] - ref.f_r).max() < 1e-10
        assert inb.sum() > 0 and np.abs(ref.f_v[inb, 0]).max() > 0
        assert max(e.values()) < ACC_TOL, (n, e)
    sim.close()


def test_womersley_inflow_rejected_without_its_parameters():
    case = fc.venous_valve(seed=2, wo=5.0, DH=2e-3, L_H=4.0)
    sim = Simulation(2, params=[__import__("paper_1911_13255_gb300")._case_params(case)])
    with pytest.raises(SphError):
        sim.set_inflow(1, 2, case.inflow_width, 0.0, case.inflow_H, case.inflow_U, 0.0, 0.0, 5.0)
    with pytest.raises(SphError):
        sim.set_inflow(1, 4, case.inflow_width, 0.0, case.inflow_H, case.inflow_U, 0.0)
    sim.set_inflow(1, 2, case.inflow_width, 0.0, case.inflow_H, case.inflow_U, 0.0, 0.6, 5.0)
    sim.close()

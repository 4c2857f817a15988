"""Single-time-step baselines through the C-ABI on the GPU, against the
oracle: the step chosen by the Section 2.2 criterion (mode "single") or by
min(dt_ac, dt_S) (mode "single_solid") from the previous step's maxima, one
solid sub-step per step, and the state after the step; a batch applies the
mode to each instance with its own maxima."""
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
MODES = {"single": 1, "single_solid": 2}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _cases():
    return [fc.tiny_box(seed=4), fc.tiny_box(seed=5, with_solid=False), fc.channel_flag(seed=6)]


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("which", [0, 1, 2])
def test_single_step_matches_oracle(mode, which):
    case = _cases()[which]
    ref = O.OracleSim(case)
    sim = Simulation.from_case(case)
    sim.set_time_stepping(mode)
    for n in range(2):
        sim.step(0.0)
        sim.sync()
        info = sim.info()
        if n == 0:   # maxima of the initial state, no acceleration yet
            want = ref.single_dt(MODES[mode])
        else:        # the previous step's FP32 maxima, as the library keeps them
            want = ref.single_dt(MODES[mode], prev["vmax_f"], prev["vmax_s"], prev["amax_s"])
        assert info["last_K"] == 1
        assert abs(info["last_dt"] - want) <= 1e-6 * want, (n, info["last_dt"], want)
        ref.step(info["last_dt"], 1)
        g = sim.get_fluid()
        e = {"dvdt": rel(g["dvdt"], ref.f_dvdt), "drho": rel(g["drho"], ref.f_drho), "v": rel(g["v"], ref.f_v)}
        assert np.abs(g["r"] - ref.f_r).max() < 1e-9
        if case.ns:
            s = sim.get_solid()
            e["fF"] = rel(s["fF"], ref.s_fF)
            e["F-I"] = rel(s["F"] - np.eye(2), ref.s_F - np.eye(2))
            e["vbar"] = rel(s["vbar"], ref.s_vbar)
        assert max(e.values()) < ACC_TOL, (n, e)
        prev = info
    sim.close()


def test_modes_order_and_return_to_multiple():
    """On the flag channel (c_S > c_F) the single step is smaller than the
    fluid step of the multiple-time-step scheme, which then takes K > 1
    sub-steps; switching back restores that scheme."""
    case = fc.channel_flag(seed=7)
    dts = {}
    for mode in ("multiple", "single", "single_solid"):
        sim = Simulation.from_case(case)
        sim.set_time_stepping(mode)
        sim.step(0.0)
        sim.sync()
        dts[mode] = (sim.info()["last_dt"], sim.info()["last_K"])
        sim.close()
    assert dts["multiple"][1] > 1
    assert dts["single"][1] == dts["single_solid"][1] == 1
    assert dts["single"][0] <= dts["single_solid"][0] < dts["multiple"][0]
    sim = Simulation.from_case(case)
    sim.set_time_stepping("single")
    sim.set_substeps(0)
    sim.step(0.0)
    sim.sync()
    assert (sim.info()["last_dt"], sim.info()["last_K"]) == dts["multiple"]
    with pytest.raises(SphError):
        sim.set_time_stepping(3)
    sim.close()


def test_batch_applies_the_mode_per_instance():
    cases = _cases()
    batch = Simulation.from_cases(cases)
    batch.set_time_stepping("single")
    batch.run(2)
    batch.sync()
    for b, case in enumerate(cases):
        single = Simulation.from_case(case)
        single.set_time_stepping("single")
        single.run(2)
        single.sync()
        got, want = batch.select(b).info(), single.info()
        assert got["last_K"] == 1
        assert got["last_dt"] == want["last_dt"], (b, got["last_dt"], want["last_dt"])
        g, w = batch.get_fluid(), single.get_fluid()
        for k in ("r", "v", "drho"):
            assert np.array_equal(g[k], w[k]), (b, k)
        single.close()
    batch.close()

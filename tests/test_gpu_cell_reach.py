"""Cells of edge >= h_F (cell_reach 2: the 5^d cells around a particle's cell)
against the oracle and against the default cells of edge >= 2 h_F, through the
C-ABI on the GPU: the same neighbour sets bit for bit, the same step to the
pair-loop tolerance, and the launch shapes that need 2 h_F cells refused."""
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

CASES = {
    "tiny_box": lambda: fc.tiny_box(seed=1),
    "tiny_box_3d": lambda: fc.tiny_box_3d(seed=1),
    "channel_flag": lambda: fc.channel_flag(seed=0),
    "dam_gate": lambda: fc.dam_gate(seed=0, dpF=0.002),
}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _reach2(name):
    case = CASES[name]()
    case.cell_reach = 2
    return case


@pytest.mark.parametrize("name", list(CASES))
def test_neighbor_sets_equal_the_default_cells(name):
    a = Simulation.from_case(CASES[name]())
    b = Simulation.from_case(_reach2(name))
    which = [0, 1] + ([2, 3] if b.ns else [])
    for _ in range(2):
        for w in which:
            pa, ia = a.debug_neighbors(w)
            pb, ib = b.debug_neighbors(w)
            assert np.array_equal(pa, pb) and np.array_equal(ia, ib), (name, w)
        for sim in (a, b):
            for _ in range(3):
                sim.step(0.0)
            sim.sync()


@pytest.mark.parametrize("lanes,compact", [(4, 0), (8, 1), (2, 1)])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_parity(name, lanes, compact):
    case = _reach2(name)
    if case.dim == 3 and lanes == 2:
        lanes = 16
    ref = O.OracleSim(case)
    dt, _, dts = ref.suggest_dt()
    K = ref.substeps(dt, dts)
    sim = Simulation.from_case(case)
    assert sim.tuning()["rows"] == 0 and sim.tuning()["tile"] == 0
    sim.set_tuning(lanes, 128, 0, compact, 0)
    sim.set_substeps(K)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    g = sim.get_fluid()
    e = {"dvdt": rel(g["dvdt"], ref.f_dvdt), "drho": rel(g["drho"], ref.f_drho), "v": rel(g["v"], ref.f_v),
         "rho-rho0": rel(g["rho"] - case.f_rho0, ref.f_rho - case.f_rho0)}
    if case.ns:
        e["fF"] = rel(sim.get_solid()["fF"], ref.s_fF)
    assert max(e.values()) < ACC_TOL, e


def test_reinitialisation_steps_agree_with_the_default_cells():
    """tiny_box reinitialises every third step (double-float number density,
    cell offsets of up to two edges)."""
    a = Simulation.from_case(CASES["tiny_box"]())
    b = Simulation.from_case(_reach2("tiny_box"))
    for _ in range(7):
        a.step(0.0)
        b.step(0.0)
    a.sync()
    b.sync()
    ga, gb = a.get_fluid(), b.get_fluid()
    assert rel(gb["drho"], ga["drho"]) < ACC_TOL
    assert rel(gb["v"], ga["v"]) < ACC_TOL


def test_row_form_and_tiles_refused():
    sim = Simulation.from_case(_reach2("channel_flag"))
    with pytest.raises(SphError):
        sim.set_tuning(4, 128, 0, 1, 0, 0, 1)
    with pytest.raises(SphError):
        sim.set_tuning(4, 128, 0, 1, 1, 0, 0)

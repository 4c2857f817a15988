"""Degenerate and ragged inputs through the C-ABI on the GPU, against the
oracle: fluid alone, fluid with walls and no body, a single fluid particle,
particles outside the cell-grid box (clamped into the border cells), an
instance without fluid neighbours for its body, and a non-finite state,
which the step reports instead of propagating silently."""
import copy

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


def _step_parity(case):
    ref = O.OracleSim(case)
    dt, _, dts = ref.suggest_dt()
    K = ref.substeps(dt, dts) if case.ns else 1
    sim = Simulation.from_case(case)
    sim.set_substeps(K)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    g = sim.get_fluid()
    e = {"dvdt": rel(g["dvdt"], ref.f_dvdt), "drho": rel(g["drho"], ref.f_drho), "v": rel(g["v"], ref.f_v)}
    assert np.abs(g["r"] - ref.f_r).max() < 1e-9
    if case.ns:
        e["fF"] = rel(sim.get_solid()["fF"], ref.s_fF)
    assert max(e.values()) < ACC_TOL, e
    return sim


def _sets_equal_oracle(sim, case):
    g = sim.get_fluid()
    P = O.make_params(case)
    rc = 2 * 1.3 * case.f_dp
    want = {0: O.pairs(P, g["r"], g["r"], rc, 1, brute=True)}
    if case.nw:
        want[1] = O.pairs(P, g["r"], case.w_r, rc, 0, brute=True)
    for which, (p, i) in want.items():
        gp, gi = sim.debug_neighbors(which)
        assert np.array_equal(gp, p) and np.array_equal(gi, i), which


def test_fluid_alone():
    case = fc.tiny_box(seed=1, with_solid=False, with_walls=False)
    assert case.ns == 0 and case.nw == 0
    _sets_equal_oracle(_step_parity(case), case)


def test_fluid_and_walls_without_a_body():
    case = fc.tiny_box(seed=2, with_solid=False)
    assert case.ns == 0 and case.nw > 0
    _sets_equal_oracle(_step_parity(case), case)


def test_a_single_fluid_particle():
    case = fc.tiny_box(seed=3, with_solid=False)
    k = len(case.f_r) // 2
    case.f_r, case.f_v, case.f_p = case.f_r[k:k + 1], case.f_v[k:k + 1], case.f_p[k:k + 1]
    assert case.nf == 1
    _sets_equal_oracle(_step_parity(case), case)


def test_particles_outside_the_grid_box_are_binned_into_border_cells():
    case = fc.tiny_box(seed=4)
    lo, hi = np.asarray(case.domain_lo, float), np.asarray(case.domain_hi, float)
    fr = np.asarray(case.f_r)
    # shrink the box so that a band of fluid lies beyond its upper x and y faces
    hi2 = hi.copy()
    hi2[0] = lo[0] + 0.6 * (fr[:, 0].max() - lo[0])
    hi2[1] = lo[1] + 0.7 * (fr[:, 1].max() - lo[1])
    case.domain_hi = tuple(hi2)
    assert (fr[:, 0] > hi2[0]).any() and (fr[:, 1] > hi2[1]).any()
    _sets_equal_oracle(_step_parity(case), case)


def test_batch_with_a_fluid_only_and_a_single_particle_instance():
    a = fc.tiny_box(seed=5, with_solid=False, with_walls=False)
    b = fc.tiny_box(seed=6)
    c = fc.tiny_box(seed=7, with_solid=False)
    k = len(c.f_r) // 3
    c.f_r, c.f_v, c.f_p = c.f_r[k:k + 1], c.f_v[k:k + 1], c.f_p[k:k + 1]
    cases = [a, b, c]
    batch = Simulation.from_cases(cases)
    for _ in range(3):
        batch.step(0.0)
    batch.sync()
    for i, case in enumerate(cases):
        single = Simulation.from_case(case)
        for _ in range(3):
            single.step(0.0)
        single.sync()
        want, got = single.get_fluid(), batch.select(i).get_fluid()
        for key in want:
            assert np.array_equal(got[key], want[key]), (i, key)
        single.close()
    batch.close()


def test_a_non_finite_state_is_reported():
    case = fc.tiny_box(seed=8)
    sim = Simulation.from_case(case)
    sim.step(0.0)
    sim.sync()
    v = sim.get_fluid()["v"].astype(np.float64)
    v[len(v) // 2, 0] = np.nan
    sim.set_fluid_state(v=v)
    sim.step(1e-5)
    with pytest.raises(SphError):
        sim.sync()
    assert sim.info()["status"] != 0


@pytest.mark.parametrize("how", ["nan", "faster_than_c0"])
def test_a_run_away_state_stops_the_context_until_a_checkpoint_is_restored(how):
    """A step that ends non-finite, or with a fluid particle faster than c0,
    stops the context: steps enqueued after it do no work (the step counter
    stays), later steps are refused, and restoring a checkpoint taken before
    lets the context step again to the same result as before."""
    case = fc.tiny_box(seed=8)
    sim = Simulation.from_case(case)
    sim.step(0.0)
    sim.sync()
    blob = sim.get_state()
    sim.step(0.0)
    sim.sync()
    ref = sim.get_fluid()
    sim.set_state(blob)
    v = sim.get_fluid()["v"].astype(np.float64)
    v[len(v) // 2, 0] = np.nan if how == "nan" else 2.0 * case.f_c0
    sim.set_fluid_state(v=v)
    sim.step(0.0)
    sim.run(3, 0.0)   # enqueued before the sync that reports the run-away
    with pytest.raises(SphError) as e:
        sim.sync()
    assert e.value.code == -5
    assert sim.info()["status"] != 0
    assert sim.info()["step"] == 2   # the run-away step completed; the three after it did nothing
    with pytest.raises(SphError) as e:
        sim.step(0.0)
    assert e.value.code == -5
    with pytest.raises(SphError):
        sim.run(1, 0.0)
    sim.set_state(blob)
    sim.step(0.0)
    sim.sync()
    g = sim.get_fluid()
    assert sim.info()["step"] == 2 and sim.info()["status"] == 0
    assert np.array_equal(g["v"], ref["v"]) and np.array_equal(g["r"], ref["r"])
    sim.close()


def test_coincident_particles():
    """A fluid particle on top of another and one on top of a solid particle:
    the pair has no direction and adds nothing on either side (the oracle's
    rule, the limit of close pairs); the step stays finite and equals the
    oracle's."""
    case = fc.tiny_box(seed=11)
    k, m = len(case.f_r) // 3, len(case.s_r0) // 2
    case.f_r = np.concatenate([case.f_r, case.f_r[k:k + 1], case.s_r0[m:m + 1]])
    case.f_v = np.concatenate([case.f_v, case.f_v[k:k + 1], case.s_v0[m:m + 1]])
    case.f_p = np.concatenate([case.f_p, case.f_p[k:k + 1], [0.0]])
    sim = _step_parity(case)
    g = sim.get_fluid()
    assert np.all(np.isfinite(g["dvdt"])) and np.all(np.isfinite(g["drho"]))
    assert np.array_equal(g["dvdt"][k], g["dvdt"][-2])   # the twins feel the same
    sim.close()

"""Neighbour rows (sphfsi_tuning.list = 1): the candidate tests run once per
rebuild and the pair loops stream each target's row.  Checked through the
C-ABI against the oracle (one step, per-step tolerance), against the cell
form (the same in-support pairs: equal pair counts), with a clump of
particles whose rows overflow (those targets fall back to the cell visit),
and with the held configuration of Algorithm 1 (rows built once per
advection step)."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import Simulation  # noqa: E402

ACC_TOL = 1e-5
CASES = {
    "tiny_box": lambda: fc.tiny_box(seed=0),
    "tiny_box_3d": lambda: fc.tiny_box_3d(seed=0),
    "channel_flag": lambda: fc.channel_flag(seed=0),
    "dam_gate": lambda: fc.dam_gate(seed=0),
}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _dt_K(ref):
    dt, _, dts = ref.suggest_dt()
    return dt, ref.substeps(dt, dts)


def _run(case, dt, K, lanes, list_on, steps=1, cadence=1):
    sim = Simulation.from_case(case)
    sim.set_tuning(lanes, 128, compact=0, rows=0, list=list_on)
    sim.set_substeps(K)
    sim.set_advection_cadence(cadence)
    out = []
    for _ in range(steps):
        sim.step(dt)
        sim.sync()
        out.append((sim.get_fluid(), sim.get_solid(), sim.info()))
    sim.close()
    return out


def _compare(case, g, s, ref):
    e = {"dvdt": rel(g["dvdt"], ref.f_dvdt), "drho": rel(g["drho"], ref.f_drho), "v": rel(g["v"], ref.f_v)}
    if case.ns:
        e["fF"] = rel(s["fF"], ref.s_fF)
        e["v_s"] = rel(s["v"], ref.s_v)
    return e


@pytest.mark.parametrize("name", list(CASES))
def test_rows_one_step_against_the_oracle_and_the_cell_form(name):
    case = CASES[name]()
    ref = O.OracleSim(case)
    dt, K = _dt_K(ref)
    ref.step(dt, K)
    lanes = 4 if case.dim == 2 else 8
    (g, s, info), = _run(case, dt, K, lanes, 1)
    (gc, sc, infoc), = _run(case, dt, K, lanes, 0)
    e = _compare(case, g, s, ref)
    print(name, {k: f"{v:.1e}" for k, v in e.items()})
    assert max(e.values()) < ACC_TOL, e
    for k in ("pairs_ff", "pairs_fw", "pairs_fs", "pairs_sf"):
        assert info[k] == infoc[k], k
    assert info["kernels_per_step"] == infoc["kernels_per_step"] + 1
    # the two forms differ only in the order of each particle's pair sums
    assert rel(g["dvdt"], gc["dvdt"]) < 1e-6


def _clumped():
    """tiny_box with 90 extra fluid particles inside 0.4 dp of one particle:
    their rows (at most 64 entries in 2-D) overflow."""
    c = fc.tiny_box(seed=4)
    rng = np.random.default_rng(9)
    k = len(c.f_r) // 2
    extra = c.f_r[k] + rng.uniform(-0.4, 0.4, size=(90, 2)) * c.f_dp
    c.f_r = np.concatenate([c.f_r, extra])
    c.f_v = np.concatenate([c.f_v, np.repeat(c.f_v[k:k + 1], 90, 0)])
    c.f_p = np.concatenate([c.f_p, np.repeat(c.f_p[k:k + 1], 90, 0)])
    c.n_reinit = 0
    return c


def test_overflowing_rows_fall_back_to_the_cell_visit():
    case = _clumped()
    ref = O.OracleSim(case)
    dt, K = _dt_K(ref)
    ref.step(dt, K)
    pairs = ref.last["n_ff"]
    (g, s, info), = _run(case, dt, K, 4, 1)
    (gc, _, infoc), = _run(case, dt, K, 4, 0)
    e = _compare(case, g, s, ref)
    print("clump", {k: f"{v:.1e}" for k, v in e.items()}, pairs)
    assert max(e.values()) < ACC_TOL, e
    assert info["pairs_ff"] == infoc["pairs_ff"] == pairs
    assert rel(g["dvdt"], gc["dvdt"]) < 1e-6


@pytest.mark.parametrize("name", ["tiny_box", "channel_flag"])
def test_rows_with_the_held_configuration_match_the_oracle(name):
    case = CASES[name]()
    n = 3
    ref = O.OracleSim(case)
    ref.set_advection_cadence(n)
    dt, K = _dt_K(ref)
    r_start = np.array(ref.f_r)
    outs = _run(case, dt, K, 4, 1, steps=2 * n + 1, cadence=n)
    for k, (g, s, info) in enumerate(outs):
        ref.step(dt, K)
        e = _compare(case, g, s, ref)
        d = g["r"] - r_start
        dr = ref.f_r - r_start
        if case.periodic_x:
            d[:, 0] -= case.Lx * np.round(d[:, 0] / case.Lx)
            dr[:, 0] -= case.Lx * np.round(dr[:, 0] / case.Lx)
        e["dr"] = rel(d, dr)
        print(name, k, {q: f"{v:.1e}" for q, v in e.items()})
        assert max(e.values()) < ACC_TOL, (k, e)
        assert info["pairs_ff"] == ref.last["n_ff"] and info["pairs_fw"] == ref.last["n_fw"]


@pytest.mark.parametrize("list_lanes", [1, 8])
def test_rows_in_a_batch_equal_single_instances_bitwise(list_lanes):
    """Rows in a batch of uneven instances (a cell's instance is found from
    its first particle; every row indexes its own instance's slots) give,
    instance by instance, the bits of one context per instance with rows."""
    cases = [fc.tiny_box(seed=2), fc.channel_flag(seed=1), fc.tiny_box(seed=3, nx=10, ny=14)]
    stream = torch.cuda.Stream()

    def shaped(sim):
        sim.set_tuning(4, 128, compact=0, rows=0, list=1, list_lanes=list_lanes)
        return sim

    batch = shaped(Simulation.from_cases(cases, stream=stream))
    for _ in range(6):
        batch.step(0.0)
    batch.sync()
    for b, case in enumerate(cases):
        single = shaped(Simulation.from_case(case, stream=stream))
        for _ in range(6):
            single.step(0.0)
        single.sync()
        got = batch.select(b)
        for x, y in ((got.get_fluid(), single.get_fluid()), (got.get_solid(), single.get_solid())):
            for k in x:
                assert np.array_equal(x[k], y[k]), (b, k)
        single.close()
    batch.close()

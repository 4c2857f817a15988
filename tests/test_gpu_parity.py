"""GPU (CUDA library, through the C-ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances: neighbour sets bit-exact (FP64 in-support test on both sides);
per-step accelerations and rates within 1e-5 relative L2 (the FP32 pair-loop
budget); positions within their FP64 drift from FP32 velocities.
"""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _csr_equal(p1, i1, p2, i2):
    return np.array_equal(np.asarray(p1), np.asarray(p2)) and np.array_equal(np.asarray(i1), np.asarray(i2))


CASES = {
    "tiny_box": lambda: fc.tiny_box(seed=1),
    "tiny_box_3d": lambda: fc.tiny_box_3d(seed=1),
    "floating_block": lambda: fc.floating_block(seed=1),
    "channel_flag": lambda: fc.channel_flag(seed=0),
    "dam_gate": lambda: fc.dam_gate(seed=0),
}


def _oracle_sets(case, f_r, s_r):
    P = O.make_params(case)
    rc = 2 * 1.3 * case.f_dp
    out = {0: O.pairs(P, f_r, f_r, rc, 1)}
    if case.nw:
        out[1] = O.pairs(P, f_r, case.w_r, rc, 0)
    if case.ns:
        out[2] = O.pairs(P, f_r, s_r, rc, 0)
        out[3] = O.pairs(P, s_r, f_r, rc, 0)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_neighbor_sets_bit_exact(name):
    case = CASES[name]()
    sim = Simulation.from_case(case)
    ref = O.OracleSim(case)
    dt, K = _dt_K(ref)
    sim.set_substeps(K)
    for stage in range(2):
        g, s = sim.get_fluid(), sim.get_solid()
        want = _oracle_sets(case, g["r"], s["r"] if case.ns else np.zeros((0, case.dim)))
        for which, (p, i) in want.items():
            gp, gi = sim.debug_neighbors(which)
            assert _csr_equal(gp, gi, p, i), (name, stage, which)
        for _ in range(3):
            sim.step(dt)
        sim.sync()


def _dt_K(ref):
    """The paper's criteria at the initial state (Eqs. dt-relax, dts-advection)."""
    dt, _, dts = ref.suggest_dt()
    return dt, ref.substeps(dt, dts)


def _one_step(case, solid_path=0):
    ref = O.OracleSim(case)
    dt, K = _dt_K(ref)
    sim = Simulation.from_case(case)
    sim.set_solid_path(solid_path)
    sim.set_substeps(K)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    return sim, ref, dt


@pytest.mark.parametrize("solid_path", [0, 1, 2], ids=["auto", "cluster_lanes", "grid"])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_parity(name, solid_path):
    case = CASES[name]()
    s_r_start = np.array(case.s_r0, dtype=np.float64)
    sim, ref, dt = _one_step(case, solid_path)
    if case.ns:
        assert sim.info()["solid_path"] == (2 if solid_path == 2 else 1)
    g, s = sim.get_fluid(), sim.get_solid()
    e = {
        "dvdt": rel(g["dvdt"], ref.f_dvdt),
        "drho": rel(g["drho"], ref.f_drho),
        "v": rel(g["v"], ref.f_v),
        "rho-rho0": rel(g["rho"] - case.f_rho0, ref.f_rho - case.f_rho0),
    }
    dr = np.abs(g["r"] - ref.f_r).max()
    if case.ns:
        e["fF"] = rel(s["fF"], ref.s_fF)
        e["v_s"] = rel(s["v"], ref.s_v) if np.linalg.norm(ref.s_v) > 0 else 0.0
        e["F-I"] = rel(s["F"] - np.eye(case.dim), ref.s_F - np.eye(case.dim))
        e["abar"] = rel(s["abar"], ref.s_abar)
        e["dr_s"] = rel(s["r"] - s_r_start, ref.s_r - s_r_start)
    print(name, {k: f"{v:.2e}" for k, v in e.items()})
    assert e["dvdt"] < ACC_TOL and e["drho"] < ACC_TOL, e
    assert e["v"] < ACC_TOL
    assert dr < 1e-9, dr
    if case.ns:
        assert e["fF"] < ACC_TOL, e
        assert e["v_s"] < ACC_TOL and e["abar"] < ACC_TOL and e["F-I"] < ACC_TOL, e
        assert e["dr_s"] < ACC_TOL, e


@pytest.mark.parametrize("name", ["tiny_box", "channel_flag", "dam_gate"])
def test_step_parity_at_evolved_state(name):
    """Run the GPU some steps, load its state into the oracle, compare one step."""
    case = CASES[name]()
    ref = O.OracleSim(case)
    dt, K = _dt_K(ref)
    sim = Simulation.from_case(case)
    sim.set_substeps(K)
    for _ in range(20):
        sim.step(dt)
    sim.sync()
    g, s = sim.get_fluid(), sim.get_solid()
    st = dict(f_r=g["r"], f_v=g["v"], f_rho=g["rho"], f_drho=g["drho"], t=sim.info()["t"], step_index=20)
    if case.ns:
        st.update(s_r=s["r"], s_v=s["v"], s_F=s["F"], s_vbar=s["vbar"], s_abar=s["abar"], s_nrm=s["nrm"])
    ref.load_state(st)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    g2, s2 = sim.get_fluid(), sim.get_solid()
    e = dict(dvdt=rel(g2["dvdt"], ref.f_dvdt), drho=rel(g2["drho"], ref.f_drho))
    if case.ns:
        e["fF"] = rel(s2["fF"], ref.s_fF)
        e["v_s"] = rel(s2["v"], ref.s_v)
    print(name, {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) < ACC_TOL, e


def test_fsi_momentum_balance_and_conservation():
    case = fc.floating_block(seed=3)
    sim = Simulation.from_case(case)
    sim.set_substeps(3)
    ref = O.OracleSim(case)
    dt, _, _ = ref.suggest_dt()
    mF, mS = case.f_rho0 * case.f_dp ** 2, case.s_rho0 * case.s_dp ** 2
    g, s = sim.get_fluid(), sim.get_solid()
    P0 = mF * g["v"].astype(np.float64).sum(0) + mS * s["v"].astype(np.float64).sum(0)
    scale = mF * np.abs(g["v"]).sum() + mS * np.abs(s["v"]).sum()
    for _ in range(50):
        sim.step(dt)
        info = sim.info()
        tot = info["mom_fs_fluid"] + info["mom_fs_solid"]
        mag = np.abs(info["mom_fs_fluid"]).max()
        assert np.abs(tot).max() <= 1e-5 * max(mag, 1e-30), (tot, mag)
    g, s = sim.get_fluid(), sim.get_solid()
    P1 = mF * g["v"].astype(np.float64).sum(0) + mS * s["v"].astype(np.float64).sum(0)
    assert np.abs(P1 - P0).max() < 1e-5 * scale


def test_deterministic_and_graph_equals_steps():
    case = fc.tiny_box(seed=5)
    ref = O.OracleSim(case)
    dt, _, _ = ref.suggest_dt()
    outs = []
    for mode in ("step", "step", "graph"):
        stream = torch.cuda.Stream()
        sim = Simulation.from_case(case, stream=stream)
        sim.set_substeps(2)
        if mode == "graph":
            sim.run(25, dt)
        else:
            for _ in range(25):
                sim.step(dt)
        sim.sync()
        g, s = sim.get_fluid(), sim.get_solid()
        outs.append((g["r"], g["v"], g["rho"], s["r"], s["v"]))
        sim.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_auto_dt_and_substeps_follow_the_criteria():
    case = fc.dam_gate(seed=0, dpF=0.002)
    sim = Simulation.from_case(case)
    sim.step(0.0)
    sim.step(0.0)
    info = sim.info()
    hF, hS = 1.3 * case.f_dp, 1.3 * case.s_dp
    cS = np.sqrt(case.s_E / (3 * (1 - 2 * case.s_nu)) / case.s_rho0)
    vmax_prev = info["vmax_f"]   # loose check: the step uses the previous step's max
    assert 0.6 * hF / (case.f_c0 + 10.0) < info["last_dt"] <= 0.6 * hF / case.f_c0 * (1 + 1e-12)
    dts = 0.6 * hS / (cS + info["vmax_s"])
    assert abs(info["last_K"] - (np.floor(info["last_dt"] / dts) + 1)) <= 1
    assert vmax_prev >= 0


@pytest.mark.parametrize("dpF", [0.002, 0.001], ids=["half_resolution", "workload_resolution"])
def test_gate_tip_parity_1000_steps(dpF):
    """Dam break through the elastic gate (at half resolution, and at the
    workload's 1 mm with 14k fluid and 1.6k solid particles): the gate-tip
    displacement after 1000 fluid steps matches the oracle within 1e-3
    (relative to max(|u|, 0.01 dp_S))."""
    case = fc.dam_gate(seed=0, dpF=dpF)
    ref = O.OracleSim(case, threaded=True)
    dt, _, dts = ref.suggest_dt(vmax_f=0.0)
    K = ref.substeps(dt, dts)
    sim = Simulation.from_case(case)
    sim.set_substeps(K)
    for _ in range(1000):
        sim.step(dt)
    sim.sync()
    for _ in range(1000):
        ref.step(dt, K)
    s = sim.get_solid()
    tip = case.tip
    u_g = s["r"][tip] - case.s_r0[tip]
    u_o = ref.s_r[tip] - case.s_r0[tip]
    err = np.linalg.norm(u_g - u_o) / max(np.linalg.norm(u_o), 0.01 * case.s_dp)
    print("tip u oracle", u_o, "gpu", u_g, "rel err", err)
    assert np.linalg.norm(u_o) > 0.1 * case.s_dp   # the gate moved
    assert err < 1e-3

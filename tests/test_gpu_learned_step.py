"""The learned solid sub-stepper inside the coupled step (GPU, through the
C-ABI) against the oracle: a rejected proposal leaves the plain path bit for
bit; an accepted one commits the network's step (oracle network on the same
features and graph) and its residual is the oracle's momentum-balance
residual; a network trained on plain steps learns them."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O
from oracle import mpnn as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import Simulation, learn  # noqa: E402

SCALES = np.array([1e-4, 1e-2, 1e-5, 5e-4, 1e-6, 1e-4, 1e-3])


def _sc():
    return dict(s_u=SCALES[0], s_v=SCALES[1], s_f=SCALES[2], s_t=SCALES[3], s_du=SCALES[4], s_dv=SCALES[5],
                s_H=SCALES[6])


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_rejected_learned_steps_leave_the_plain_path_bitwise():
    case = fc.channel_flag(seed=0)
    a, b = Simulation.from_case(case), Simulation.from_case(case)
    b.set_learned(learn.init_params(2, 0), SCALES, tol=0.0)
    for _ in range(10):
        a.step(0.0)
        b.step(0.0)
    a.sync()
    b.sync()
    for ga, gb in ((a.get_fluid(), b.get_fluid()), (a.get_solid(), b.get_solid())):
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), k
    ib = b.info()
    assert ib["learned_rejected"] == 10 and ib["learned_accepted"] == 0 and ib["learned_residual"] > 0


def test_accepted_step_applies_the_network_and_matches_the_oracle_residual():
    case = fc.channel_flag(seed=0)
    d = case.dim
    sim = Simulation.from_case(case)
    for _ in range(5):
        sim.step(0.0)
    sim.sync()
    pre = sim.get_solid()
    theta = learn.init_params(2, 3)
    sim.set_learned(theta, SCALES, tol=1e30)
    sim.step(0.0)
    sim.sync()
    post, info = sim.get_solid(), sim.info()
    assert info["learned_accepted"] == 1
    dt, fF = info["last_dt"], post["fF"].astype(np.float64)
    cons = np.asarray(case.s_cons)
    free = cons == 0
    m = case.s_rho0 * case.s_dp ** d
    graph = M.build_graph(case.s_r0, case.s_dp, d)   # the oracle's own graph, not the library's
    x = M.features(pre["r"] - case.s_r0, pre["v"], pre["F"] - np.eye(d), fF, cons, dt, _sc(), d)
    x = x.astype(np.float32).astype(np.float64)
    y, _ = M.forward(theta.astype(np.float64), x, graph, d, round_bf16=True)
    du, dv = M.apply_outputs(y, pre["v"].astype(np.float64), fF, cons, dt, m, case.gravity, _sc(), d)
    e_du = rel((post["r"] - pre["r"])[free], du[free])
    e_dv = rel((post["v"].astype(np.float64) - pre["v"])[free], dv[free])
    print("du", e_du, "dv", e_dv)
    assert e_du < 2e-3 and e_dv < 2e-3
    assert np.array_equal(post["r"][~free], pre["r"][~free])
    # the residual with the oracle's F(x) and force loop at the mid positions
    ref = O.OracleSim(case)
    ref.set_solid_positions(pre["r"] + 0.5 * (post["r"] - pre["r"]))
    F_mid = ref.F_from_positions()
    ref.s_fF[:] = fF
    acc = ref.solid_accel(F_mid)
    vn = post["v"].astype(np.float64)
    e = (vn - pre["v"])[free] - dt * acc[free]
    R = np.linalg.norm(e) / np.linalg.norm(vn[free])
    print("R", info["learned_residual"], R)
    assert info["learned_residual"] == pytest.approx(R, rel=1e-2)
    # committed F is F of the new positions; time averages are the step's changes
    ref.set_solid_positions(post["r"])
    assert rel(post["F"] - np.eye(d), ref.F_from_positions() - np.eye(d)) < 1e-4
    assert rel(post["vbar"][free], ((post["r"] - pre["r"]) / dt)[free]) < 1e-12


@pytest.mark.parametrize("name", ["channel_flag", "tiny_box_3d"])
def test_library_graph_equals_the_oracle_graph(name):
    """sphfsi_solid_graph (the device's static list and V0 grad0 W entries)
    against the oracle's brute-force graph: same rows and columns, w and g
    equal to FP32 rounding."""
    case = getattr(fc, name)(seed=0)
    sim = Simulation.from_case(case)
    ptr, idx, w, g = sim.solid_graph()
    optr, oidx, ow, og = M.build_graph(case.s_r0, case.s_dp, case.dim)
    assert np.array_equal(ptr, optr) and np.array_equal(idx, oidx)
    assert np.abs(w - ow).max() <= 1e-12 * np.abs(ow).max()
    assert np.abs(g - og).max() <= 1e-6 * np.abs(og).max()
    sim.close()


def test_in_step_features_equal_the_training_features():
    """The feature rows the step's kernel feeds the network equal the rows
    learn.features builds on the host from the same state (the state before
    the step, the step's coupling force and dt), to FP32 rounding, so that
    the network is trained on inputs laid out and scaled as in a step."""
    case = fc.channel_flag(seed=0)
    d = case.dim
    sim = Simulation.from_case(case)
    for _ in range(5):
        sim.step(0.0)
    sim.sync()
    pre = sim.get_solid()
    sim.set_learned(learn.init_params(d, 1), SCALES, tol=0.0)   # proposals rejected: the plain step runs
    sim.step(0.0)
    sim.sync()
    post, info = sim.get_solid(), sim.info()
    x_gpu = sim.learned_features()
    data = {"u": (pre["r"] - case.s_r0)[None], "v": pre["v"].astype(np.float64)[None],
            "H": (pre["F"] - np.eye(d)).reshape(1, case.ns, d * d), "f": post["fF"].astype(np.float64)[None],
            "dt": np.array([info["last_dt"]])}
    x_host = learn.features(data, 0, case.s_cons, SCALES)
    nf = 2 * d + d * d + d + 2
    assert np.all(x_gpu[:, nf:] == 0.0) and np.all(x_host[:, nf:] == 0.0)
    for lo, hi in ((0, d), (d, 2 * d), (2 * d, 2 * d + d * d), (2 * d + d * d, 3 * d + d * d), (nf - 2, nf)):
        a, b = x_gpu[:, lo:hi].astype(np.float64), x_host[:, lo:hi].astype(np.float64)
        assert np.abs(a - b).max() <= 1e-6 * max(np.abs(b).max(), 1e-30), (lo, hi)
    sim.close()


def test_a_network_trained_on_plain_steps_learns_them():
    case = fc.channel_flag(seed=0)
    d = case.dim
    cons = np.asarray(case.s_cons)
    m = case.s_rho0 * case.s_dp ** d
    sim = Simulation.from_case(case)
    data = learn.collect(sim, 80, case.s_r0)
    graph = sim.solid_graph()
    scales = learn.scales_from(data, m, case.gravity, cons)
    theta, losses = learn.train(graph, d, data, cons, m, case.gravity, scales, iters=400, replicas=16, lr=1e-3)
    print("loss", losses[:10].mean(), losses[-10:].mean())
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.3 * losses[:20].mean()
    # the trained network's step from a recorded state, against the plain step
    plain = Simulation.from_case(case)
    learned = Simulation.from_case(case)
    for _ in range(60):
        plain.step(0.0)
        learned.step(0.0)
    learned.set_learned(theta, scales, tol=1e30)
    pre = plain.get_solid()
    plain.step(0.0)
    learned.step(0.0)
    a, b = plain.get_solid(), learned.get_solid()
    free = cons == 0
    du_plain = (a["r"] - pre["r"])[free]
    err = rel((b["r"] - pre["r"])[free], du_plain)
    # what the network adds: the explicit predictor it corrects (du = dt v)
    # against the same plain step
    err_pred = rel(plain.info()["last_dt"] * pre["v"][free].astype(np.float64), du_plain)
    print("one-step displacement error: learned", err, "explicit predictor", err_pred,
          "residual", learned.info()["learned_residual"])
    assert err < 0.1 and err < 0.5 * err_pred

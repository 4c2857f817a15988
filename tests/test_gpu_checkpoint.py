"""Checkpoint blobs and the time-step criteria through the C-ABI on the GPU:
a restored state continues bit for bit like the original, into the same or
a freshly built context; a blob of another configuration is refused; the
suggested steps equal the oracle's criteria at the initial state."""
import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1911_13255_gb300 import Simulation, SphError  # noqa: E402


def _snapshot(sim):
    out = {f"f_{k}": v for k, v in sim.get_fluid().items()}
    if sim.ns:
        out.update({f"s_{k}": v for k, v in sim.get_solid().items()})
    i = sim.info()
    out.update(t=np.array([i["t"]]), step=np.array([i["step"]]), pairs=np.array([i["pairs_total"]]))
    return out


def _equal(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("name", ["dam_gate", "channel_flag"])
def test_restored_state_continues_bit_for_bit(name):
    case = {"dam_gate": lambda: fc.dam_gate(seed=0, dpF=0.002), "channel_flag": lambda: fc.channel_flag(seed=0)}[name]()
    sim = Simulation.from_case(case)
    for _ in range(5):
        sim.step(0.0)
    blob = sim.get_state()
    for _ in range(6):
        sim.step(0.0)
    sim.sync()
    want = _snapshot(sim)
    sim.set_state(blob)
    for _ in range(6):
        sim.step(0.0)
    sim.sync()
    _equal(want, _snapshot(sim))
    fresh = Simulation.from_case(case)
    fresh.set_state(blob)
    for _ in range(6):
        fresh.step(0.0)
    fresh.sync()
    _equal(want, _snapshot(fresh))


def test_blob_of_another_configuration_is_refused():
    a = Simulation.from_case(fc.tiny_box(seed=1))
    b = Simulation.from_case(fc.channel_flag(seed=0))
    blob = a.get_state()
    before = _snapshot(b)
    with pytest.raises(SphError):
        b.set_state(blob)
    with pytest.raises(SphError):
        a.set_state(blob[:-8])
    _equal(before, _snapshot(b))


@pytest.mark.parametrize("name", ["dam_gate", "channel_flag", "tiny_box"])
def test_suggested_steps_follow_the_oracle_criteria(name):
    case = {"dam_gate": lambda: fc.dam_gate(seed=0, dpF=0.002), "channel_flag": lambda: fc.channel_flag(seed=0),
            "tiny_box": lambda: fc.tiny_box(seed=1)}[name]()
    sim = Simulation.from_case(case)
    ref = O.OracleSim(case)
    vf = float(np.float32(np.sqrt((np.asarray(case.f_v) ** 2).sum(1)).max())) if case.nf else 0.0
    vs = float(np.float32(np.sqrt((np.asarray(case.s_v0) ** 2).sum(1)).max())) if case.ns else 0.0
    want = ref.suggest_dt(vf, vs, 0.0)
    got = sim.suggest_dt()
    for g, w in zip(got[:2], want[:2]):
        assert g == pytest.approx(w, rel=1e-6)
    if case.ns:
        assert got[2] == pytest.approx(want[2], rel=1e-6)
    sim.step(0.0)
    sim.sync()
    assert sim.info()["last_dt"] == pytest.approx(got[0], rel=1e-12)

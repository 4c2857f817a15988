"""Batched contexts: independent instances of uneven size, advanced by the same
launches, give instance by instance the same bits as one context per
instance, and a batch member matches the FP64 oracle like a single problem.

The batch mixes what the per-instance look-ups must keep apart: channels with
flags of different sizes and materials (uneven K), a tank without a solid, a
periodic blob without walls, and a walled box with a free block.
"""
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


def _mixed_cases():
    cases = fc.flag_batch(seed=7, n=4, nf_lo=2000, nf_hi=9000)
    cases.insert(1, fc.hydrostatic_column(seed=2))
    cases.append(fc.floating_block(seed=4))
    cases.append(fc.tiny_box(seed=6))
    return cases


def _state(sim):
    g = sim.get_fluid()
    out = {f"f_{k}": v for k, v in g.items()}
    if sim.ns:
        out.update({f"s_{k}": v for k, v in sim.get_solid().items()})
    info = sim.info()
    for k in ("t", "step", "last_dt", "last_K", "pairs_ff", "pairs_fw", "pairs_fs", "pairs_sf", "pairs_ss",
              "pairs_total", "vmax_f", "vmax_s"):
        out[k] = np.asarray(info[k])
    return out


@pytest.mark.parametrize("mode", ["step", "graph"])
def test_batch_equals_single_instances_bitwise(mode):
    cases = _mixed_cases()
    nsteps = 12
    stream = torch.cuda.Stream()
    batch = Simulation.from_cases(cases, stream=stream)
    assert batch.n_instances == len(cases)
    if mode == "graph":
        batch.run(nsteps, 0.0)
    else:
        for _ in range(nsteps):
            batch.step(0.0)
    batch.sync()
    Ks = []
    total = 0
    for b, case in enumerate(cases):
        single = Simulation.from_case(case, stream=stream)
        for _ in range(nsteps):
            single.step(0.0)
        single.sync()
        want = _state(single)
        got = _state(batch.select(b))
        assert set(want) == set(got)
        for k in want:
            assert np.array_equal(got[k], want[k]), (b, case.name, k)
        Ks.append(int(want["last_K"]))
        total += int(want["pairs_total"])
        single.close()
    assert batch.pairs_total() == total
    # the flags' materials differ, so do their sub-step counts
    flag_K = [K for K, c in zip(Ks, cases) if c.name.startswith("flag_batch")]
    assert len(set(flag_K)) > 1, flag_K
    batch.close()


def test_batch_member_parity_with_oracle():
    cases = _mixed_cases()
    batch = Simulation.from_cases(cases)
    batch.step(0.0)
    batch.sync()
    for b in (0, 1, len(cases) - 2):
        case = cases[b]
        info = batch.select(b).info()
        ref = O.OracleSim(case)
        dt_ref, _, dts = ref.suggest_dt()
        assert abs(info["last_dt"] - dt_ref) <= 1e-6 * dt_ref
        if case.ns:
            assert info["last_K"] == ref.substeps(info["last_dt"], dts)
        ref.step(info["last_dt"], max(info["last_K"], 1))
        g = batch.get_fluid()
        e = dict(dvdt=rel(g["dvdt"], ref.f_dvdt), drho=rel(g["drho"], ref.f_drho), v=rel(g["v"], ref.f_v))
        if case.ns:
            s = batch.get_solid()
            e["fF"] = rel(s["fF"], ref.s_fF)
            e["F-I"] = rel(s["F"] - np.eye(2), ref.s_F - np.eye(2))
            e["abar"] = rel(s["abar"], ref.s_abar)
        print(case.name, {k: f"{v:.2e}" for k, v in e.items()})
        assert max(e.values()) < ACC_TOL, (case.name, e)
    batch.close()


def test_batch_neighbor_sets_bit_exact_per_instance():
    cases = _mixed_cases()[:3]
    batch = Simulation.from_cases(cases)
    for b, case in enumerate(cases):
        batch.select(b)
        P = O.make_params(case)
        rc = 2 * 1.3 * case.f_dp
        f_r = batch.get_fluid()["r"]
        want = {0: O.pairs(P, f_r, f_r, rc, 1)}
        if case.nw:
            want[1] = O.pairs(P, f_r, case.w_r, rc, 0)
        if case.ns:
            s_r = batch.get_solid()["r"]
            want[2] = O.pairs(P, f_r, s_r, rc, 0)
            want[3] = O.pairs(P, s_r, f_r, rc, 0)
        for which, (p, i) in want.items():
            gp, gi = batch.debug_neighbors(which)
            assert np.array_equal(gp, p) and np.array_equal(gi, i), (b, which)
    batch.close()


def test_batch_rejects_bad_selection_and_grid_path():
    cases = _mixed_cases()[:2]
    batch = Simulation.from_cases(cases)
    with pytest.raises(SphError):
        batch.select(len(cases))
    with pytest.raises(SphError):
        batch.set_solid_path(2)
    batch.close()


@pytest.mark.parametrize("name,lanes,block,compact,tile,records,rows", [
    ("channel_flag", 2, 64, 1, 0, 0, 1), ("channel_flag", 4, 128, 0, 0, 1, 0), ("channel_flag", 8, 256, 1, 0, 1, 0),
    ("channel_flag", 8, 128, 0, 0, 0, 1), ("tiny_box_3d", 4, 128, 0, 0, 1, 1), ("tiny_box_3d", 16, 256, 1, 0, 0, 0),
    ("tiny_box_3d", 8, 64, 1, 0, 1, 1), ("channel_flag", 4, 128, 1, 1, 0, 0), ("channel_flag", 2, 256, 0, 1, 1, 0),
    ("tiny_box_3d", 4, 128, 0, 1, 0, 0), ("tiny_box_3d", 8, 64, 1, 1, 1, 0), ("dam_gate", 4, 128, 1, 1, 1, 0),
    ("dam_gate", 4, 128, 1, 0, 0, 1), ("dam_gate", 8, 128, 1, 0, 1, 0), ("tiny_box_3d", 16, 128, 0, 0, 0, 1),
    ("dam_gate", 8, 128, 0, 0, 2, 1), ("tiny_box_3d", 8, 128, 1, 0, 2, 0), ("channel_flag", 4, 64, 1, 1, 2, 0)])
def test_every_launch_shape_matches_the_oracle(name, lanes, block, compact, tile, records, rows):
    """Each compiled lane count, block size, pair-loop form, tile mode, records form and cell-visit form
    computes the same step."""
    case = {"channel_flag": lambda: fc.channel_flag(seed=0), "tiny_box_3d": lambda: fc.tiny_box_3d(seed=1),
            "dam_gate": lambda: fc.dam_gate(seed=0, dpF=0.002)}[name]()
    ref = O.OracleSim(case)
    dt, _, dts = ref.suggest_dt()
    K = ref.substeps(dt, dts)
    sim = Simulation.from_case(case)
    sim.set_tuning(lanes, block, 0, compact, tile, records, rows)
    t = sim.tuning()
    assert (t["lanes"], t["block"], t["compact"], t["tile"], t["records"], t["rows"]) == \
        (lanes, block, compact, tile, records, rows)
    sim.set_substeps(K)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    g, s = sim.get_fluid(), sim.get_solid()
    e = dict(dvdt=rel(g["dvdt"], ref.f_dvdt), drho=rel(g["drho"], ref.f_drho), fF=rel(s["fF"], ref.s_fF))
    assert max(e.values()) < ACC_TOL, e
    with pytest.raises(SphError):
        sim.set_tuning(4 if case.dim == 2 else 8, 128, 0, 1, 1, 0, 1)   # rows with tiles
    with pytest.raises(SphError):
        sim.set_tuning(3, 128)
    with pytest.raises(SphError):
        sim.set_tuning(4 if case.dim == 2 else 8, 96)


def test_autotune_leaves_the_state_unchanged_and_keeps_parity():
    cases = _mixed_cases()
    stream = torch.cuda.Stream()
    batch = Simulation.from_cases(cases, stream=stream)
    for _ in range(3):
        batch.step(0.0)
    batch.sync()
    before = [_state(batch.select(b)) for b in range(len(cases))]
    best = batch.autotune(0.0, steps=3)
    assert best["step_ms"] > 0 and best["lanes"] in (2, 4, 8) and best["block"] in (64, 128, 256)
    assert batch.tuning()["lanes"] == best["lanes"]
    after = [_state(batch.select(b)) for b in range(len(cases))]
    for b in range(len(cases)):
        for k in before[b]:
            assert np.array_equal(before[b][k], after[b][k]), (b, k)
    # the tuned batch keeps stepping like the default one, to rounding
    ref = Simulation.from_cases(cases, stream=stream)
    for _ in range(3):
        ref.step(0.0)
    for sim in (batch, ref):
        sim.run(5, 0.0)
        sim.sync()
    for b in range(len(cases)):
        g, h = batch.select(b).get_fluid(), ref.select(b).get_fluid()
        assert rel(g["r"], h["r"]) < 1e-9 and rel(g["v"], h["v"]) < 1e-4
    batch.close()
    ref.close()


@pytest.mark.parametrize("name", ["dam_gate", "channel_flag", "floating_block"])
def test_two_thread_solid_kernel_matches_the_oracle(name):
    """The 2-D cluster sub-step kernel with two threads per particle."""
    case = {"dam_gate": lambda: fc.dam_gate(seed=0), "channel_flag": lambda: fc.channel_flag(seed=0),
            "floating_block": lambda: fc.floating_block(seed=1)}[name]()
    ref = O.OracleSim(case)
    dt, _, dts = ref.suggest_dt()
    K = ref.substeps(dt, dts)
    sim = Simulation.from_case(case)
    sim.set_tuning(4, 128, 2)
    assert sim.tuning()["solid_variant"] == 2
    sim.set_substeps(K)
    s_r0 = np.array(case.s_r0)
    sim.step(dt)
    sim.sync()
    ref.step(dt, K)
    s = sim.get_solid()
    e = dict(v=rel(s["v"], ref.s_v), F=rel(s["F"] - np.eye(2), ref.s_F - np.eye(2)), abar=rel(s["abar"], ref.s_abar),
             dr=rel(s["r"] - s_r0, ref.s_r - s_r0))
    assert max(e.values()) < ACC_TOL, e


def test_two_thread_solid_kernel_batch_equals_single():
    cases = _mixed_cases()
    batch = Simulation.from_cases(cases)
    batch.set_tuning(4, 128, 2)
    for _ in range(6):
        batch.step(0.0)
    batch.sync()
    for b, case in enumerate(cases):
        single = Simulation.from_case(case)
        single.set_tuning(4, 128, 2)
        for _ in range(6):
            single.step(0.0)
        single.sync()
        if case.ns:
            want, got = single.get_solid(), batch.select(b).get_solid()
            for k in want:
                assert np.array_equal(got[k], want[k]), (b, k)
        single.close()
    batch.close()


@pytest.mark.parametrize("name", ["dam_gate", "channel_flag", "floating_block"])
def test_solid_push_and_pull_forms_are_bitwise_equal(name):
    """Variants 0 and 4 read neighbours from the CTA's own halo copies (refreshed with
    stores ordered by cluster barriers, or with asynchronous stores counted on mbarriers),
    variant 3 from the owning CTAs across the cluster, variant 5 evolves the halo
    particles' stresses in every CTA that reads them (one cluster barrier per sub-step):
    the same values in the same order, so the same bits."""
    case = {"dam_gate": lambda: fc.dam_gate(seed=0), "channel_flag": lambda: fc.channel_flag(seed=0),
            "floating_block": lambda: fc.floating_block(seed=1)}[name]()
    sims = []
    for variant in (0, 3, 4, 5):
        sim = Simulation.from_case(case)
        sim.set_tuning(4, 128, variant)
        for _ in range(4):
            sim.step(0.0)
        sim.sync()
        sims.append(sim)
    assert sims[3].info()["solid_path"] == 3   # the one-barrier form ran
    a = sims[0].get_solid()
    for other in sims[1:]:
        b = other.get_solid()
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert sims[0].info()["solid_path"] == 1
    assert all(sim.info()["status"] == 0 for sim in sims)


@pytest.mark.parametrize("name", ["dam_gate", "tiny_box_3d"])
def test_binning_forms_are_bitwise_equal(name):
    """The three binning forms (four kernels with records from the cell groups, the same with
    records per slot, one cooperative kernel) produce the same records, hence the same steps."""
    case = {"dam_gate": lambda: fc.dam_gate(seed=0), "tiny_box_3d": lambda: fc.tiny_box_3d(seed=1)}[name]()
    states = []
    for records in (0, 1, 2):
        sim = Simulation.from_case(case)
        t = sim.tuning()
        sim.set_tuning(t["lanes"], t["block"], t["solid_variant"], t["compact"], t["tile"], records, t["rows"])
        assert sim.tuning()["records"] == records
        for _ in range(5):
            sim.step(0.0)
        sim.sync()
        states.append((sim.get_fluid(), sim.get_solid() if case.ns else {}))
    for fl, so in states[1:]:
        for k in states[0][0]:
            assert np.array_equal(fl[k], states[0][0][k]), k
        for k in states[0][1]:
            assert np.array_equal(so[k], states[0][1][k]), k


def test_fused_binning_batch_equals_single():
    """A batch stepped with the cooperative binning kernel matches its instances stepped alone."""
    cases = _mixed_cases()
    batch = Simulation.from_cases(cases)
    t = batch.tuning()
    batch.set_tuning(t["lanes"], t["block"], 0, t["compact"], 0, 2, t["rows"])
    for _ in range(4):
        batch.step(0.0)
    batch.sync()
    for b, case in enumerate(cases):
        single = Simulation.from_case(case)
        single.set_tuning(t["lanes"], t["block"], 0, t["compact"], 0, 0, t["rows"])
        for _ in range(4):
            single.step(0.0)
        single.sync()
        want, got = single.get_fluid(), batch.select(b).get_fluid()
        for k in want:
            assert np.array_equal(got[k], want[k]), (b, k)
        single.close()
    batch.close()


def test_solid_position_reads_all_and_async_agree_per_step():
    """The solid positions of a batch read after each graph-replayed step:
    without waiting (enqueued on the stream into pinned buffers, read back
    one step later, after an event) they are, bit for bit, the rows the
    waiting read gives and each instance's own positions, step by step."""
    cases = _mixed_cases()
    stream = torch.cuda.Stream()
    a = Simulation.from_cases(cases, stream=stream)
    b = Simulation.from_cases(cases, stream=stream)
    dim = cases[0].dim
    n = sum(c.ns for c in cases)
    bufs = [torch.empty((n, dim), dtype=torch.float64).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    want = np.zeros((n, dim))
    prev = None
    for k in range(6):
        a.run(1, 0.0)
        a.get_solid_positions_async(bufs[k % 2])
        evs[k % 2].record(stream)
        b.run(1, 0.0)
        b.get_solid_positions_all(want)
        rows = np.concatenate([b.select(i).get_solid()["r"] for i in range(len(cases))])
        assert np.array_equal(want, rows), k
        if prev is not None:
            evs[(k - 1) % 2].synchronize()
            assert np.array_equal(bufs[(k - 1) % 2].numpy(), prev), k - 1
        prev = want.copy()
    a.sync()
    assert np.array_equal(bufs[5 % 2].numpy(), prev)
    a.close()
    b.close()

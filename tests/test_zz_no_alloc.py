"""The allocation-free entry point sphfsi_neighbor_counts_noalloc, called
through the C-ABI, gives the same per-particle neighbour counts as the
context-based sphfsi_debug_neighbors and as the oracle's neighbour lists
(integer counts: exact), on two calls in a row with different inputs, and
for points given outside a periodic x range.

It serves callers that cannot call cudaMalloc (for example code that only
receives input/output buffers from a framework whose caching allocator owns
the device memory); its scratch is a fixed file-scope device array shared by
all calls.  This file is collected last so that a failure here stops a
first-failure run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import fsi_cases as fc
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1911_13255_gb300 as pkg  # noqa: E402


def _params(case):
    p = pkg.Params()
    p.dim, p.periodic_x, p.x_lo, p.Lx = case.dim, case.periodic_x, case.x_lo, case.Lx
    p.free_surface, p.n_reinit = case.free_surface, case.n_reinit
    for k in range(3):
        p.gravity[k] = case.gravity[k]
        p.domain_lo[k] = case.domain_lo[k]
        p.domain_hi[k] = case.domain_hi[k]
    return p


def _reference_counts(case):
    sim = pkg.Simulation.from_case(case)
    ptr, _ = sim.debug_neighbors(0)
    sim.close()
    return np.diff(ptr).astype(np.int32)


def _noalloc_counts(case, stream):
    r = torch.from_numpy(np.ascontiguousarray(case.f_r, dtype=np.float64)).cuda()
    counts = torch.full((case.nf,), -1, dtype=torch.int32, device="cuda")
    p = _params(case)
    rc = pkg.lib().sphfsi_neighbor_counts_noalloc(ctypes.byref(p), case.nf, r.data_ptr(), case.f_dp,
                                                  counts.data_ptr(), stream.cuda_stream)
    assert rc == 0, pkg.lib().sphfsi_strerror(rc)
    stream.synchronize()
    return counts.cpu().numpy()


def _oracle_counts(case):
    ptr, _ = O.pairs(case, case.f_r, case.f_r, 2.0 * (1.3 * case.f_dp), same=True)
    return np.diff(ptr).astype(np.int32)


def test_noalloc_neighbor_counts_match_context_entry_point_twice():
    stream = torch.cuda.Stream()
    for case in (fc.channel_flag(seed=0), fc.tiny_box_3d(seed=2)):
        want = _reference_counts(case)
        got = _noalloc_counts(case, stream)
        assert np.array_equal(got, want)
        assert np.array_equal(got, _oracle_counts(case))
        assert want.sum() > 0


def test_noalloc_counts_points_given_outside_the_period():
    """Periodic x: shifting points by whole periods does not change their
    neighbours; the counts equal the oracle's on the points inside."""
    stream = torch.cuda.Stream()
    case = fc.channel_flag(seed=1)
    assert case.periodic_x
    want = _oracle_counts(case)
    rng = np.random.default_rng(3)
    shifted = case.f_r.copy()
    shifted[:, 0] += case.Lx * rng.choice([-2.0, -1.0, 0.0, 1.0], size=case.nf)
    moved = fc.Case(**{**case.__dict__, "f_r": shifted})
    assert np.array_equal(_noalloc_counts(moved, stream), want)


def test_noalloc_rejects_oversized_input():
    case = fc.tiny_box(seed=0)
    p = _params(case)
    n = (1 << 18) + 1
    rc = pkg.lib().sphfsi_neighbor_counts_noalloc(ctypes.byref(p), n, 1, case.f_dp, 1, None)
    assert rc == -7   # SPHFSI_E_CAPACITY, checked before any device access
    # a box of more cells than the maximum (tiny dp), and non-finite sizes,
    # are rejected before any device access too
    assert pkg.lib().sphfsi_neighbor_counts_noalloc(ctypes.byref(p), 10, 1, 1e-9, 1, None) == -7
    assert pkg.lib().sphfsi_neighbor_counts_noalloc(ctypes.byref(p), 10, 1, float("inf"), 1, None) == -1
    p.domain_hi[0] = float("inf")
    assert pkg.lib().sphfsi_neighbor_counts_noalloc(ctypes.byref(p), 10, 1, case.f_dp, 1, None) == -1

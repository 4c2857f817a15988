"""Pins of the FP64 oracle of the learned sub-stepper (oracle/mpnn.py).

Each pin checks the oracle against something other than itself: central
finite differences of the loss for the backward pass, the dot-product
identity for the aggregation adjoint, permutation equivariance of the
network, torch's own bfloat16 conversion for the rounding, and the closed
form of Adam's first step.
"""
import numpy as np
import pytest

from oracle import mpnn as M


def _body(nx=6, ny=3, dp=0.01, seed=0):
    rng = np.random.default_rng(seed)
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    r0 = np.stack([xs.ravel(), ys.ravel()], 1) * dp + rng.uniform(-1e-3, 1e-3, (nx * ny, 2)) * dp
    return r0, dp


def _inputs(n, dim, rng):
    x = np.zeros((n, M.FIN))
    x[:, :M.n_features(dim)] = rng.normal(size=(n, M.n_features(dim)))
    return x


def test_graph_is_brute_force_support_and_antisymmetric_gradients():
    r0, dp = _body()
    ptr, idx, w, g = M.build_graph(r0, dp, 2)
    h = 1.3 * dp
    n = len(r0)
    for a in range(n):
        want = [b for b in range(n) if b != a and ((r0[a] - r0[b]) ** 2).sum() < 4 * h * h]
        assert idx[ptr[a]:ptr[a + 1]].tolist() == want
    # symmetric relation, w symmetric, g antisymmetric (one body, one spacing)
    pos = {(a, int(b)): q for a in range(n) for q, b in zip(range(ptr[a], ptr[a + 1]), idx[ptr[a]:ptr[a + 1]])}
    for (a, b), q in pos.items():
        q2 = pos[(b, a)]
        assert w[q] == pytest.approx(w[q2], rel=1e-14)
        assert np.allclose(g[q], -g[q2], rtol=1e-13, atol=0)


def test_aggregation_of_a_constant_field_vanishes_and_adjoint_is_exact():
    rng = np.random.default_rng(1)
    r0, dp = _body()
    graph = M.build_graph(r0, dp, 2)
    n = len(r0)
    ms = M.aggregate(np.ones((n, M.C)) * 3.7, graph)
    assert all(np.abs(m).max() == 0.0 for m in ms)
    h = rng.normal(size=(n, M.C))
    dms = [rng.normal(size=(n, M.C)) for _ in range(3)]
    lhs = sum((dm * m).sum() for dm, m in zip(dms, M.aggregate(h, graph)))
    rhs = (M.aggregate_adjoint(dms, graph) * h).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    dim = 2
    r0, dp = _body(5, 3)
    graph = M.build_graph(r0, dp, dim)
    n = len(r0)
    theta = M.init_params(dim, seed=3) * 0.5
    theta += rng.normal(scale=1e-2, size=theta.shape)
    x = _inputs(n, dim, rng)
    t = rng.normal(size=(n, M.NOUT))
    mask = rng.uniform(size=n) > 0.2

    def L(th):
        out, _ = M.forward(th, x, graph, dim, round_bf16=False)
        return M.loss(out, t, mask, dim)[0]

    out, cache = M.forward(theta, x, graph, dim, round_bf16=False)
    _, dout = M.loss(out, t, mask, dim)
    grad = M.backward(theta, cache, dout, graph, dim, round_bf16=False)
    # a spread of entries from every tensor
    o, picks = 0, []
    for name, s in M.param_shapes(dim):
        k = int(np.prod(s))
        picks += list(o + rng.choice(k, size=min(6, k), replace=False))
        o += k
    eps = 1e-6
    for i in picks:
        e = np.zeros_like(theta)
        e[i] = eps
        fd = (L(theta + e) - L(theta - e)) / (2 * eps)
        assert fd == pytest.approx(grad[i], rel=2e-5, abs=1e-9), (i, fd, grad[i])


def test_network_is_permutation_equivariant():
    rng = np.random.default_rng(4)
    dim = 2
    r0, dp = _body(6, 4)
    n = len(r0)
    perm = rng.permutation(n)
    theta = M.init_params(dim, seed=5)
    theta += rng.normal(scale=1e-2, size=theta.shape)
    x = _inputs(n, dim, rng)
    out, _ = M.forward(theta, x, M.build_graph(r0, dp, dim), dim, round_bf16=False)
    out_p, _ = M.forward(theta, x[perm], M.build_graph(r0[perm], dp, dim), dim, round_bf16=False)
    assert np.allclose(out_p, out[perm], rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0, 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)
    assert M.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie to even
    assert M.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(7)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    th1, m, v = M.adam(theta, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    assert np.allclose(th1, theta - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_outputs_and_targets_are_inverse():
    rng = np.random.default_rng(8)
    dim, n = 2, 30
    sc = dict(s_u=1e-3, s_v=1e-2, s_f=1e-4, s_t=1e-3, s_du=1e-6, s_dv=1e-4, s_H=1e-3)
    v, f = rng.normal(size=(n, dim)), rng.normal(size=(n, dim))
    cons = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    du, dv = rng.normal(size=(n, dim)), rng.normal(size=(n, dim))
    t = M.targets(du, dv, v, f, cons, 1e-3, 2.5e-4, (0.0, -9.81, 0.0), sc, dim)
    du2, dv2 = M.apply_outputs(t, v, f, cons, 1e-3, 2.5e-4, (0.0, -9.81, 0.0), sc, dim)
    free = cons == 0
    assert np.allclose(du2[free], du[free], rtol=1e-12, atol=1e-18)
    assert np.allclose(dv2[free], dv[free], rtol=1e-12, atol=1e-15)
    assert np.abs(du2[~free]).max() == 0.0 and np.abs(dv2[~free]).max() == 0.0

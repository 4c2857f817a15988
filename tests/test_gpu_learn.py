"""Learned sub-stepper kernels on the GPU against the FP64 oracle
(oracle/mpnn.py) and against FP64 products of the same bfloat16 operands."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1911_13255_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 128, 64), (256, 128, 128), (384, 512, 512),
                                   (128, 64, 192), (256, 32, 1024), (1280, 48, 64), (512, 640, 256),
                                   (256, 256, 320), (128, 512, 8192), (128, 16, 4160)])
def test_gemm_matches_fp64_products_of_the_bf16_operands(M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    C = pkg.gemm_bf16(A.cuda(), B.cuda(), bias.cuda())
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T + bias.double()
    err = (C.cpu().double() - ref).norm() / ref.norm()
    # FP32 accumulation over K: about sqrt(K) roundings of 2^-24 relative
    assert err < 4.0 * np.sqrt(K) * 2.0 ** -24, float(err)
    assert pkg.tc_status(reset=True) == 0


def test_gemm_rejects_unpadded_shapes():
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pkg.SphError):
        pkg.gemm_bf16(A, B)
    A = torch.zeros(128, 48, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 48, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pkg.SphError):
        pkg.gemm_bf16(A, B)


# ---------------------------------------------------------------------------
# the network against the oracle (oracle/mpnn.py, bf16 rounding at the GEMM
# operands, FP64 elsewhere)
# ---------------------------------------------------------------------------
from oracle import mpnn as M  # noqa: E402

# Tolerances: the GPU evaluates graph sums, activations and the residual
# stream in FP32 and accumulates GEMMs in FP32; both sides round the GEMM
# operands to bfloat16 at the same points, so the difference is FP32
# rounding plus rare one-ulp bfloat16 flips where an FP32 value sits at a
# rounding tie of the FP64 one (each worth 2^-8 of one operand).
FWD_TOL = 2e-3
GRAD_TOL = 5e-3


def _body(dim, shape, dp=0.01, seed=0):
    rng = np.random.default_rng(seed)
    axes = np.meshgrid(*[np.arange(k) for k in shape], indexing="ij")
    r0 = np.stack([a.ravel() for a in axes], 1) * dp
    return r0 + rng.uniform(-1e-3, 1e-3, r0.shape) * dp, dp


def _net_case(dim, shape, R, seed):
    rng = np.random.default_rng(seed)
    r0, dp = _body(dim, shape, seed=seed)
    graph = M.build_graph(r0, dp, dim)
    theta = M.init_params(dim, seed=seed)
    theta = theta + rng.normal(scale=0.02, size=theta.shape)        # non-zero biases too
    theta = theta.astype(np.float32).astype(np.float64)
    n = len(r0)
    x = np.zeros((R * n, M.FIN))
    x[:, :M.n_features(dim)] = rng.normal(size=(R * n, M.n_features(dim)))
    x = x.astype(np.float32).astype(np.float64)
    return graph, theta, x, n


def _oracle_fwd(theta, x, graph, dim, n, R):
    outs, caches = [], []
    for r in range(R):
        o, c = M.forward(theta, x[r * n:(r + 1) * n], graph, dim, round_bf16=True)
        outs.append(o)
        caches.append(c)
    return np.concatenate(outs), caches


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dim,shape,R", [(2, (14, 5), 1), (2, (9, 6), 5), (3, (5, 4, 3), 2)])
def test_mpnn_forward_matches_oracle(dim, shape, R):
    graph, theta, x, n = _net_case(dim, shape, R, seed=dim + R)
    net = pkg.Mpnn(dim, graph, replicas=R)
    assert net.n_params == M.n_params(dim)
    net.set_params(theta)
    out = net.forward(x)
    want, _ = _oracle_fwd(theta, x, graph, dim, n, R)
    e = rel(out, want)
    print("forward rel err", e)
    assert e < FWD_TOL, e
    assert np.allclose(net.get_params(), theta.astype(np.float32))
    net.close()


@pytest.mark.parametrize("dim,shape,R", [(2, (12, 5), 3), (3, (5, 4, 3), 1)])
def test_mpnn_backward_matches_oracle(dim, shape, R):
    graph, theta, x, n = _net_case(dim, shape, R, seed=10 + dim)
    rng = np.random.default_rng(3)
    dout = rng.normal(size=(R * n, M.NOUT)).astype(np.float32).astype(np.float64)
    net = pkg.Mpnn(dim, graph, replicas=R)
    net.set_params(theta)
    net.forward(x)
    grad = net.backward(dout)
    _, caches = _oracle_fwd(theta, x, graph, dim, n, R)
    want = sum(M.backward(theta, caches[r], dout[r * n:(r + 1) * n], graph, dim, round_bf16=True)
               for r in range(R))
    gp, wp = M.unpack(grad, dim), M.unpack(want, dim)
    errs = {k: rel(gp[k], wp[k]) for k in wp}
    print("grad rel err", {k: f"{v:.1e}" for k, v in errs.items()})
    assert max(errs.values()) < GRAD_TOL, errs
    net.close()


def test_mpnn_training_step_matches_oracle_and_learns():
    dim, R = 2, 4
    graph, theta, x, n = _net_case(dim, (10, 4), R, seed=21)
    rng = np.random.default_rng(5)
    # a smooth target: a fixed random linear map of the features
    Wt = rng.normal(size=(M.FIN, M.NOUT)) * 0.3
    t = np.tanh(x @ Wt).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=R * n) > 0.25).astype(np.uint8)
    net = pkg.Mpnn(dim, graph, replicas=R)
    net.set_params(theta)
    L0 = net.train_step(x, t, mask, lr=1e-3)
    # the oracle's loss at the same parameters
    out, caches = _oracle_fwd(theta, x, graph, dim, n, R)
    L_ref, _ = M.loss(out, t, mask, dim)
    assert L0 == pytest.approx(L_ref, rel=FWD_TOL)
    losses = [L0] + [net.train_step(x, t, mask, lr=1e-3) for _ in range(150)]
    print("loss", losses[0], losses[50], losses[-1])
    assert losses[-1] < 0.2 * losses[0]
    net.close()


def test_mpnn_rejects_an_asymmetric_graph():
    r0, dp = _body(2, (5, 4))
    ptr, idx, w, g = M.build_graph(r0, dp, 2)
    g2 = g.copy()
    g2[0] *= 2.0
    with pytest.raises(pkg.SphError):
        pkg.Mpnn(2, (ptr, idx, w, g2))

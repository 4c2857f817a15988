"""FP64 oracle of the learned solid sub-stepper (message-passing network).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the benchmark's CPU
legs, never by the product package; shares no code with the CUDA path.

The paper integrates the solid with K sub-steps per fluid step (Section 3.3).
The learned form replaces those K sub-steps of one fluid step by one
evaluation of a network over the body's static neighbour graph (the same
reference-configuration neighbour list the sub-steps use, support 2 h_S),
and keeps the plain sub-stepping as fallback and as the measure of its error.  This module states
that network in plain numpy, FP64, node by node and layer by layer:

  features   x_a = [u_a / s_u, v_a / s_v, H_a / s_H, f_a / s_f, c_a, dt / s_t, 0...]
             u = r - r0, H = F - I (row-major), f the fluid force of the step,
             c = 1 for a constrained particle; padded to FIN columns
  encoder    h = silu(x W_enc^T + b_enc)                        (N x 128)
  3 layers   m0_a = sum_b w_ab (h_b - h_a)
             mk_a = sum_b g_ab[k] (h_b - h_a),   k < dim
             z = [h, m0, m1, .., m_dim]                          (N x 128 (2 + dim))
             h <- h + silu(z W_l^T + b_l)
  decoder    y = h W_dec^T + b_dec                              (N x NOUT)
  outputs    du_a = dt v_a + s_du y[0:dim],  dv_a = dt (f_a / m_a + g) + s_dv y[dim:2 dim]
             (constrained particles: 0)

with the edge weights of the reference configuration w_ab = V0 W(|r0_ab|, h_S)
and g_ab = h_S V0 grad_a W(|r0_ab|, h_S) (Wendland C2, Section 2; the factor
h_S makes the gradient channels dimensionless like the partition-of-unity
weights w).

With round_bf16=True the oracle rounds to bfloat16 (round to nearest even)
exactly where the GPU kernels feed the tensor cores: the operands of every
GEMM (activations, output gradients and the weights); all other arithmetic is
FP64.  With round_bf16=False it is plain FP64 (used for the finite-difference
pins of the backward pass).
"""
from __future__ import annotations

import math

import numpy as np

C = 128          # hidden width
FIN = 64         # padded input width (GEMM K granularity)
NOUT = 16        # padded output width (smallest tensor-core N)
LAYERS = 3


def zdim(dim):
    return C * (2 + dim)


def n_features(dim):
    """Meaningful input columns: u, v, H, f, c, dt."""
    return dim + dim + dim * dim + dim + 1 + 1


def param_shapes(dim):
    """Flat parameter vector layout: weights [out, in] row-major, then bias."""
    shp = [("enc_W", (C, FIN)), ("enc_b", (C,))]
    for l in range(LAYERS):
        shp += [(f"W{l}", (C, zdim(dim))), (f"b{l}", (C,))]
    shp += [("dec_W", (NOUT, C)), ("dec_b", (NOUT,))]
    return shp


def n_params(dim):
    return sum(int(np.prod(s)) for _, s in param_shapes(dim))


def unpack(theta, dim):
    out, o = {}, 0
    for name, s in param_shapes(dim):
        n = int(np.prod(s))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(s)
        o += n
    return out


def pack(parts, dim):
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in param_shapes(dim)])


def init_params(dim, seed=0):
    """He-style uniform init; biases zero; decoder scaled down (small initial correction)."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, s in param_shapes(dim):
        if name.endswith("_b") or name.startswith("b"):
            parts[name] = np.zeros(s)
        else:
            fan_in = s[1]
            lim = math.sqrt(6.0 / fan_in) * (0.1 if name == "dec_W" else 1.0)
            parts[name] = rng.uniform(-lim, lim, s)
    return pack(parts, dim)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) via FP32, returned as FP64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, on):
    return bf16(x) if on else x


def silu(y):
    return y / (1.0 + np.exp(-y))


def dsilu(y):
    s = 1.0 / (1.0 + np.exp(-y))
    return s + y * s * (1.0 - s)


# ---------------------------------------------------------------------------
# graph
# ---------------------------------------------------------------------------
def wendland(dim, r, h):
    q = r / h
    a = np.clip(1.0 - 0.5 * q, 0.0, None)
    alpha = 7.0 / (4.0 * math.pi * h * h) if dim == 2 else 21.0 / (16.0 * math.pi * h ** 3)
    return alpha * a ** 4 * (1.0 + 2.0 * q)


def wendland_dr(dim, r, h):
    q = r / h
    a = np.clip(1.0 - 0.5 * q, 0.0, None)
    alpha = 7.0 / (4.0 * math.pi * h * h) if dim == 2 else 21.0 / (16.0 * math.pi * h ** 3)
    return -5.0 * alpha / h * q * a ** 3


def build_graph(r0, dp, dim):
    """Static neighbour graph of a body in its reference configuration:
    ordered pairs a != b with |r0_a - r0_b|^2 < (2 h_S)^2, h_S = 1.3 dp, by
    brute force; rows sorted by b.  Returns (ptr, idx, w, g)."""
    r0 = np.asarray(r0, np.float64)
    n = len(r0)
    h = 1.3 * dp
    V0 = dp ** dim
    ptr = [0]
    idx, w, g = [], [], []
    for a in range(n):
        d = r0[a] - r0
        r2 = (d * d).sum(1)
        nb = np.where((r2 < 4.0 * h * h) & (np.arange(n) != a))[0]
        r = np.sqrt(r2[nb])
        idx.extend(nb.tolist())
        w.extend((V0 * wendland(dim, r, h)).tolist())
        g.extend((h * V0 * wendland_dr(dim, r, h)[:, None] * d[nb] / r[:, None]).tolist())
        ptr.append(len(idx))
    return (np.array(ptr, np.int64), np.array(idx, np.int64), np.array(w, np.float64),
            np.array(g, np.float64).reshape(-1, dim))


def aggregate(h, graph):
    """[m0, m1, .., m_dim]: sums over each row of c_ab (h_b - h_a)."""
    ptr, idx, w, g = graph
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    diff = h[idx] - h[rows]
    coefs = [w] + [g[:, k] for k in range(g.shape[1])]
    out = []
    for c in coefs:
        m = np.zeros_like(h)
        np.add.at(m, rows, c[:, None] * diff)
        out.append(m)
    return out


def aggregate_adjoint(dms, graph):
    """Gradient of sum_k <dm_k, m_k(h)> with respect to h (plain scatter)."""
    ptr, idx, w, g = graph
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    coefs = [w] + [g[:, k] for k in range(g.shape[1])]
    dh = np.zeros_like(dms[0])
    for c, dm in zip(coefs, dms):
        t = c[:, None] * dm[rows]
        np.add.at(dh, idx, t)
        np.add.at(dh, rows, -t)
    return dh


# ---------------------------------------------------------------------------
# features and outputs
# ---------------------------------------------------------------------------
def features(u, v, H, f, cons, dt, scales, dim):
    """Input matrix (N x FIN); scales = dict(s_u, s_v, s_H, s_f, s_t)."""
    n = len(u)
    x = np.zeros((n, FIN))
    o = 0
    x[:, o:o + dim] = np.asarray(u) / scales["s_u"]; o += dim
    x[:, o:o + dim] = np.asarray(v) / scales["s_v"]; o += dim
    x[:, o:o + dim * dim] = np.asarray(H).reshape(n, dim * dim) / scales["s_H"]; o += dim * dim
    x[:, o:o + dim] = np.asarray(f) / scales["s_f"]; o += dim
    x[:, o] = np.asarray(cons, np.float64); o += 1
    x[:, o] = dt / scales["s_t"]
    return x


def apply_outputs(y, v, f, cons, dt, m, g, scales, dim):
    """(du, dv) of the step from the network outputs."""
    free = (np.asarray(cons) == 0)[:, None]
    gv = np.asarray(g, np.float64)[:dim]
    du = dt * np.asarray(v) + scales["s_du"] * y[:, :dim]
    dv = dt * (np.asarray(f) / m + gv) + scales["s_dv"] * y[:, dim:2 * dim]
    return du * free, dv * free


def targets(du, dv, v, f, cons, dt, m, g, scales, dim):
    """Inverse of apply_outputs: the outputs that reproduce (du, dv)."""
    gv = np.asarray(g, np.float64)[:dim]
    t = np.zeros((len(du), NOUT))
    t[:, :dim] = (np.asarray(du) - dt * np.asarray(v)) / scales["s_du"]
    t[:, dim:2 * dim] = (np.asarray(dv) - dt * (np.asarray(f) / m + gv)) / scales["s_dv"]
    return t


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def forward(theta, x, graph, dim, round_bf16=True):
    p = unpack(theta, dim)
    rb = round_bf16
    cache = {"x": x}
    y = _r(x, rb) @ _r(p["enc_W"], rb).T + p["enc_b"]
    cache["y_enc"] = y
    h = silu(y)
    for l in range(LAYERS):
        ms = aggregate(h, graph)
        z = np.concatenate([h] + ms, axis=1)
        cache[f"z{l}"] = z
        y = _r(z, rb) @ _r(p[f"W{l}"], rb).T + p[f"b{l}"]
        cache[f"y{l}"] = y
        h = h + silu(y)
    cache["h_out"] = h
    out = _r(h, rb) @ _r(p["dec_W"], rb).T + p["dec_b"]
    return out, cache


def loss(out, t, mask, dim):
    """Mean over unmasked particles of the squared error of the 2 dim outputs."""
    m = np.asarray(mask, np.float64)[:, None]
    cnt = max(m.sum(), 1.0)
    e = (out[:, :2 * dim] - t[:, :2 * dim]) * m
    L = (e * e).sum() / cnt
    dout = np.zeros_like(out)
    dout[:, :2 * dim] = 2.0 * e / cnt
    return L, dout


def backward(theta, cache, dout, graph, dim, round_bf16=True):
    """Gradient of <dout, out> with respect to the flat parameter vector."""
    p = unpack(theta, dim)
    rb = round_bf16
    gr = {}
    h = cache["h_out"]
    gr["dec_W"] = _r(dout, rb).T @ _r(h, rb)
    gr["dec_b"] = dout.sum(0)
    dh = _r(dout, rb) @ _r(p["dec_W"], rb)
    for l in reversed(range(LAYERS)):
        y, z = cache[f"y{l}"], cache[f"z{l}"]
        dy = dh * dsilu(y)
        gr[f"W{l}"] = _r(dy, rb).T @ _r(z, rb)
        gr[f"b{l}"] = dy.sum(0)
        dz = _r(dy, rb) @ _r(p[f"W{l}"], rb)
        dms = [dz[:, C * (k + 1):C * (k + 2)] for k in range(1 + dim)]
        dh = dh + dz[:, :C] + aggregate_adjoint(dms, graph)
    dy = dh * dsilu(cache["y_enc"])
    gr["enc_W"] = _r(dy, rb).T @ _r(cache["x"], rb)
    gr["enc_b"] = dy.sum(0)
    return pack(gr, dim)


def adam(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; step counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v

"""Training data and training loop of the learned solid sub-stepper.

The network (include/sphfsi.h, sphfsi_mpnn_*) maps one body's state at the
start of a fluid step and the step's fluid force to the displacement and
velocity change over the step.  Training pairs come from the plain method:
`collect` steps a Simulation and records, per step, the solid state before
the step, the coupling force of the step and the state after it.  `train`
fits the network with Adam on the tensor-core kernels, R samples per batch
(one network evaluation over R copies of the body graph).  Everything here is
argument marshalling around the C-ABI plus numpy bookkeeping.
"""
from __future__ import annotations

import math

import numpy as np

from . import Mpnn

FIN, NOUT = 64, 16


def n_params(dim):
    C = 128
    zd = C * (2 + dim)
    return C * FIN + C + 3 * (C * zd + C) + NOUT * C + NOUT


def init_params(dim, seed=0):
    """Uniform He initialisation of the weights (decoder scaled by 0.1), zero biases."""
    rng = np.random.default_rng(seed)
    C = 128
    zd = C * (2 + dim)
    parts = []
    for out, inp, scale in [(C, FIN, 1.0)] + [(C, zd, 1.0)] * 3 + [(NOUT, C, 0.1)]:
        lim = math.sqrt(6.0 / inp) * scale
        parts.append(rng.uniform(-lim, lim, out * inp))
        parts.append(np.zeros(out))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == n_params(dim)
    return theta


def collect(sim, steps, r0, dt=0.0):
    """Step `sim` (its selected instance) `steps` times with the plain method
    and return the per-step samples: u, v, H = F - I, f (coupling force of the
    step), dt, du, dv (arrays with a leading step axis)."""
    d = sim.dim
    rec = {k: [] for k in ("u", "v", "H", "f", "dt", "du", "dv")}
    s = sim.get_solid()
    for _ in range(steps):
        sim.step(dt)
        sim.sync()
        s1 = sim.get_solid()
        rec["u"].append(s["r"] - r0)
        rec["v"].append(s["v"].astype(np.float64))
        rec["H"].append((s["F"] - np.eye(d)).reshape(len(r0), d * d))
        rec["f"].append(s1["fF"].astype(np.float64))
        rec["dt"].append(sim.info()["last_dt"])
        rec["du"].append(s1["r"] - s["r"])
        rec["dv"].append(s1["v"].astype(np.float64) - s["v"].astype(np.float64))
        s = s1
    return {k: np.asarray(v) for k, v in rec.items()}


def scales_from(data, m, g, cons):
    """(s_u, s_v, s_f, s_t, s_du, s_dv, s_H): RMS sizes of the free
    particles' inputs and of the corrections the network has to produce."""
    free = np.asarray(cons) == 0
    dim = data["u"].shape[-1]
    gv = np.asarray(g, np.float64)[:dim]
    dt = data["dt"][:, None, None]
    ru = data["du"] - dt * data["v"]
    rv = data["dv"] - dt * (data["f"] / m + gv)

    def rms(a):
        return float(np.sqrt(np.mean(a[:, free] ** 2))) or 1.0

    return np.array([rms(data["u"]), rms(data["v"]), rms(data["f"]), float(np.mean(data["dt"])), rms(ru), rms(rv),
                     rms(data["H"])])


def features(data, k, cons, scales):
    """Input rows of step k (n x 64), laid out as the in-step feature kernel."""
    d = data["u"].shape[-1]
    n = data["u"].shape[1]
    x = np.zeros((n, FIN), np.float32)
    o = 0
    x[:, o:o + d] = data["u"][k] / scales[0]; o += d
    x[:, o:o + d] = data["v"][k] / scales[1]; o += d
    x[:, o:o + d * d] = data["H"][k] / scales[6]; o += d * d
    x[:, o:o + d] = data["f"][k] / scales[2]; o += d
    x[:, o] = np.asarray(cons, np.float32); o += 1
    x[:, o] = data["dt"][k] / scales[3]
    return x


def targets(data, k, m, g, scales):
    """Outputs that reproduce step k's (du, dv) (n x 16)."""
    d = data["u"].shape[-1]
    gv = np.asarray(g, np.float64)[:d]
    dt = data["dt"][k]
    t = np.zeros((data["u"].shape[1], NOUT), np.float32)
    t[:, :d] = (data["du"][k] - dt * data["v"][k]) / scales[4]
    t[:, d:2 * d] = (data["dv"][k] - dt * (data["f"][k] / m + gv)) / scales[5]
    return t


def train(graph, dim, data, cons, m, g, scales, iters=2000, replicas=32, lr=1e-3, seed=0, theta=None,
          stream=None, log_every=0, noise=0.0):
    """Fit the network to the recorded steps; returns (theta, losses).
    noise > 0 adds Gaussian noise of that standard deviation to the
    normalised state inputs (u, v, F - I) of every batch, so that the network
    also sees states slightly off the recorded trajectories."""
    rng = np.random.default_rng(seed)
    nsteps = data["u"].shape[0]
    R = min(replicas, nsteps)
    net = Mpnn(dim, graph, replicas=R, stream=stream)
    net.set_params(init_params(dim, seed) if theta is None else theta)
    X = np.stack([features(data, k, cons, scales) for k in range(nsteps)])
    T = np.stack([targets(data, k, m, g, scales) for k in range(nsteps)])
    mask = np.tile((np.asarray(cons) == 0).astype(np.uint8), R)
    losses = []
    for it in range(iters):
        ks = rng.choice(nsteps, size=R, replace=False)
        xb = X[ks].reshape(-1, FIN)
        if noise > 0.0:
            xb = xb.copy()
            ns = 2 * dim + dim * dim
            xb[:, :ns] += rng.normal(scale=noise, size=(xb.shape[0], ns)).astype(np.float32)
        lr_it = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))   # cosine decay
        L = net.train_step(xb, T[ks].reshape(-1, NOUT), mask, lr=max(lr_it, 1e-6))
        losses.append(L)
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {L:.3e}", flush=True)
    theta = net.get_params()
    net.close()
    return theta, np.asarray(losses)

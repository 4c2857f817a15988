"""Seeded synthetic inputs for the multi-resolution SPH FSI solver and its oracle.

This module is shared by the tests, the benchmark, the oracle driver and the
GPU binding's callers.  It holds geometry and physical constants only: lattices,
jitter, outward surface normals, constrained (clamped) flags, hydrostatic
initial pressure and the case parameters.  It contains none of the method's
arithmetic (no kernel, equation of state, Riemann solver, stress or time
integration), so both sides of every parity test compute everything from the
same raw inputs on their own.

Geometry follows the paper's benchmarks (Section 4.1, flow-induced vibration of
a flag behind a cylinder; Section 4.2, dam break through an elastic gate) at
the sizes of the workloads used here; where a figure is missing from the text,
the geometry is the one stated in each builder's docstring.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Case:
    """One FSI problem instance as raw arrays (FP64, original particle order)."""
    name: str
    dim: int
    # global parameters
    gravity: tuple
    periodic_x: int = 0
    x_lo: float = 0.0
    Lx: float = 0.0
    free_surface: int = 0
    n_reinit: int = 0
    # inflow buffer (profile 0: parabolic in y over [y0, y0+H]; 1: uniform; 2: Womersley;
    # 3: parabolic in y and in z over the duct [y0, y0+H] x [z0, z0+Hz])
    inflow_on: int = 0
    inflow_profile: int = 0
    inflow_width: float = 0.0
    inflow_y0: float = 0.0
    inflow_H: float = 1.0
    inflow_U: float = 0.0
    inflow_tramp: float = 0.0
    inflow_period: float = 0.0     # profile 2 (Womersley): period T
    inflow_wo: float = 0.0         # profile 2: Womersley number (H/2) sqrt(omega / nu)
    inflow_z0: float = 0.0         # profile 3: the duct's z range [z0, z0 + Hz]
    inflow_Hz: float = 0.0
    # bounding box for a fixed cell grid (particles outside are clamped in)
    domain_lo: tuple = (0.0, 0.0, 0.0)
    domain_hi: tuple = (1.0, 1.0, 1.0)
    # fluid
    f_r: np.ndarray = None
    f_v: np.ndarray = None
    f_p: np.ndarray = None          # initial pressure (density follows from the EoS)
    f_dp: float = 0.0
    f_rho0: float = 1.0
    f_c0: float = 1.0
    f_eta: float = 0.0
    # walls (static boundary particles)
    w_r: np.ndarray = None
    w_n: np.ndarray = None
    w_dp: float = 0.0
    # solid body
    s_r0: np.ndarray = None
    s_v0: np.ndarray = None
    s_n0: np.ndarray = None
    s_cons: np.ndarray = None       # uint8: 1 = constrained (clamped / rigid root)
    s_dp: float = 0.0
    s_rho0: float = 1.0
    s_E: float = 1.0
    s_nu: float = 0.3
    # observer: index of the tip particle (sensor S)
    tip: int = -1
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nf(self):
        return 0 if self.f_r is None else len(self.f_r)

    @property
    def nw(self):
        return 0 if self.w_r is None else len(self.w_r)

    @property
    def ns(self):
        return 0 if self.s_r0 is None else len(self.s_r0)


def _empty(dim):
    return np.zeros((0, dim))


def lattice(lo, hi, dp):
    """Cell-centred lattice points lo + (k + 1/2) dp inside [lo, hi)."""
    axes = []
    for a, b in zip(lo, hi):
        n = int(round((b - a) / dp))
        axes.append(a + (np.arange(n) + 0.5) * dp)
    grids = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grids], axis=1)


def jitter(r, dp, amp, rng):
    """Uniform jitter of amplitude amp*dp on every coordinate."""
    if amp == 0.0 or len(r) == 0:
        return r.copy()
    return r + rng.uniform(-amp, amp, size=r.shape) * dp


def _wall_layers_y(x_lo, x_hi, y_face, side, dp, layers, dim, z_lo=None, z_hi=None):
    """Wall particles below (side=-1) or above (side=+1) the plane y=y_face."""
    ys = [y_face + side * (k + 0.5) * dp for k in range(layers)]
    xs = x_lo + (np.arange(int(round((x_hi - x_lo) / dp))) + 0.5) * dp
    if dim == 2:
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        r = np.stack([X.ravel(), Y.ravel()], 1)
    else:
        zs = z_lo + (np.arange(int(round((z_hi - z_lo) / dp))) + 0.5) * dp
        X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
        r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n = np.zeros_like(r)
    n[:, 1] = -side
    return r, n


def _box_walls_2d(lo, hi, dp, layers, left=True, right=True, bottom=True, top=False):
    """Walls around [lo, hi] with outward (into the fluid) normals; corners diagonal."""
    L = layers * dp
    pts = lattice((lo[0] - L, lo[1] - L), (hi[0] + L, hi[1] + L), dp)
    x, y = pts[:, 0], pts[:, 1]
    inside = (x > lo[0]) & (x < hi[0]) & (y > lo[1]) & (y < hi[1])
    keep = ~inside
    if not left:
        keep &= ~(x < lo[0])
    if not right:
        keep &= ~(x > hi[0])
    if not bottom:
        keep &= ~(y < lo[1])
    if not top:
        keep &= ~(y > hi[1])
    pts = pts[keep]
    x, y = pts[:, 0], pts[:, 1]
    n = np.zeros_like(pts)
    n[:, 0] = np.where(x < lo[0], 1.0, np.where(x > hi[0], -1.0, 0.0))
    n[:, 1] = np.where(y < lo[1], 1.0, np.where(y > hi[1], -1.0, 0.0))
    nn = np.linalg.norm(n, axis=1)
    nn[nn == 0] = 1.0
    return pts, n / nn[:, None]


def _rect_normals(r, x0, x1, y0, y1, faces=("l", "r", "b", "t")):
    """Outward normal of the nearest face of an axis-aligned rectangle (2-D)."""
    d = {
        "l": (r[:, 0] - x0, np.array([-1.0, 0.0])),
        "r": (x1 - r[:, 0], np.array([1.0, 0.0])),
        "b": (r[:, 1] - y0, np.array([0.0, -1.0])),
        "t": (y1 - r[:, 1], np.array([0.0, 1.0])),
    }
    dist = np.stack([d[f][0] for f in faces], 1)
    k = np.argmin(dist, 1)
    dirs = np.stack([d[f][1] for f in faces], 0)
    return dirs[k]


# --------------------------------------------------------------------------
# Small test problems
# --------------------------------------------------------------------------

def tiny_box(seed=0, nx=16, ny=12, dpF=0.01, ratio=2, free_block=True, gravity=-9.81,
             jitter_amp=1e-3, c0=10.0, eta=1e-3, rho0=1.0, with_solid=True, with_walls=True):
    """2-D fluid block in a walled box with a small elastic block resting in the fluid.

    Walls: 4 layers at dp_F around three sides (open top).  The solid block sits
    inside the fluid, its left column clamped when free_block is False.
    """
    rng = np.random.default_rng(seed)
    W, H = nx * dpF, ny * dpF
    fr = lattice((0.0, 0.0), (W, H), dpF)
    dpS = dpF / ratio
    # solid block: 6*dpS wide x 4*dpS tall, centred at (0.55W, 0.45H)
    bw, bh = 4 * dpF, 2 * dpF
    bx0, by0 = 0.55 * W - bw / 2, 0.45 * H - bh / 2
    bx0 = round(bx0 / dpF) * dpF
    by0 = round(by0 / dpF) * dpF
    if with_solid:
        sr = lattice((bx0, by0), (bx0 + bw, by0 + bh), dpS)
        inside = (fr[:, 0] > bx0) & (fr[:, 0] < bx0 + bw) & (fr[:, 1] > by0) & (fr[:, 1] < by0 + bh)
        fr = fr[~inside]
        sn = _rect_normals(sr, bx0, bx0 + bw, by0, by0 + bh)
        cons = np.zeros(len(sr), np.uint8)
        if not free_block:
            cons[sr[:, 0] < bx0 + 2 * dpS] = 1
        sr = jitter(sr, dpS, jitter_amp, rng)
    else:
        sr = _empty(2)
        sn = _empty(2)
        cons = np.zeros(0, np.uint8)
    fr = jitter(fr, dpF, jitter_amp, rng)
    if with_walls:
        wr, wn = _box_walls_2d((0.0, 0.0), (W, H + 4 * dpF), dpF, 4)
    else:
        wr, wn = _empty(2), _empty(2)
    fv = rng.uniform(-0.05, 0.05, size=fr.shape)
    fp = rng.uniform(-0.5, 0.5, size=len(fr)) * rho0 * c0 * c0 * 1e-3
    sv = rng.uniform(-0.02, 0.02, size=sr.shape)
    sv[cons == 1] = 0.0
    tip = int(np.argmax(sr[:, 0])) if len(sr) else -1
    return Case(
        name="tiny_box", dim=2, gravity=(0.0, gravity, 0.0), n_reinit=3, free_surface=1,
        domain_lo=(-5 * dpF, -5 * dpF, 0.0), domain_hi=(W + 5 * dpF, H + 10 * dpF, 0.0),
        f_r=fr, f_v=fv, f_p=fp, f_dp=dpF, f_rho0=rho0, f_c0=c0, f_eta=eta,
        w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=sv, s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=10.0 * rho0, s_E=2e2, s_nu=0.4,
        tip=tip,
    )


def tiny_box_3d(seed=0, n=(8, 6, 6), dpF=0.02, ratio=2, gravity=-9.81, jitter_amp=1e-3,
                c0=10.0, eta=1e-3, rho0=1.0):
    """3-D fluid block in a box walled on the floor and four sides with a clamped plate."""
    rng = np.random.default_rng(seed)
    L = np.array(n, float) * dpF
    fr = lattice((0, 0, 0), tuple(L), dpF)
    dpS = dpF / ratio
    # plate: 2*dpF thick in x, clamped at the floor, spanning 4 dpF in z
    px0 = round(0.5 * L[0] / dpF) * dpF
    p_lo = (px0, 0.0, round(0.25 * L[2] / dpF) * dpF)
    p_hi = (px0 + 2 * dpF, 0.6 * L[1], p_lo[2] + 4 * dpF)
    p_hi = (p_hi[0], round(p_hi[1] / dpF) * dpF, p_hi[2])
    sr = lattice(p_lo, p_hi, dpS)
    inside = np.all((fr > np.array(p_lo)) & (fr < np.array(p_hi)), axis=1)
    fr = fr[~inside]
    # normals: nearest face among +-x, +y, +-z
    dists = np.stack([sr[:, 0] - p_lo[0], p_hi[0] - sr[:, 0], p_hi[1] - sr[:, 1],
                      sr[:, 2] - p_lo[2], p_hi[2] - sr[:, 2]], 1)
    dirs = np.array([[-1, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], float)
    sn = dirs[np.argmin(dists, 1)]
    cons = (sr[:, 1] < 2 * dpS).astype(np.uint8)
    sr = jitter(sr, dpS, jitter_amp, rng)
    fr = jitter(fr, dpF, jitter_amp, rng)
    # walls: 4 layers around floor and sides (open top)
    Lw = 4 * dpF
    wr = lattice((-Lw, -Lw, -Lw), (L[0] + Lw, L[1] + 2 * dpF, L[2] + Lw), dpF)
    inside = np.all((wr > 0) & (wr < np.array([L[0], L[1] + 10, L[2]])), axis=1)
    wr = wr[~inside]
    wn = np.zeros_like(wr)
    for ax in range(3):
        wn[:, ax] = np.where(wr[:, ax] < 0, 1.0, np.where((wr[:, ax] > L[ax]) & (ax != 1), -1.0, 0.0))
    wn /= np.linalg.norm(wn, axis=1)[:, None]
    fv = rng.uniform(-0.05, 0.05, size=fr.shape)
    fp = rng.uniform(-0.5, 0.5, size=len(fr)) * rho0 * c0 * c0 * 1e-3
    sv = rng.uniform(-0.02, 0.02, size=sr.shape)
    sv[cons == 1] = 0.0
    tip = int(np.argmax(sr[:, 1] + 1e-3 * sr[:, 2]))
    return Case(
        name="tiny_box_3d", dim=3, gravity=(0.0, gravity, 0.0), n_reinit=3, free_surface=1,
        domain_lo=(-6 * dpF, -6 * dpF, -6 * dpF), domain_hi=(L[0] + 6 * dpF, L[1] + 8 * dpF, L[2] + 6 * dpF),
        f_r=fr, f_v=fv, f_p=fp, f_dp=dpF, f_rho0=rho0, f_c0=c0, f_eta=eta,
        w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=sv, s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=10.0 * rho0, s_E=5e2, s_nu=0.4,
        tip=tip,
    )


def floating_block(seed=0, nx=20, ny=16, dpF=0.01, ratio=2, c0=10.0, eta=1e-3):
    """Fluid blob with an embedded free elastic block: no walls, no gravity, periodic in x.

    With no external force the total momentum of fluid plus solid is conserved
    by the pairwise-antisymmetric coupling of Section 2.2 and the position-based
    Verlet scheme of Section 3.3.
    """
    c = tiny_box(seed=seed, nx=nx, ny=ny, dpF=dpF, ratio=ratio, free_block=True, gravity=0.0,
                 c0=c0, eta=eta, with_walls=False)
    c.name = "floating_block"
    c.n_reinit = 0
    c.periodic_x = 1
    c.x_lo = 0.0
    c.Lx = nx * dpF
    c.domain_lo = (0.0, -10 * dpF, 0.0)
    c.domain_hi = (nx * dpF, ny * dpF + 10 * dpF, 0.0)
    return c


def hydrostatic_column(seed=0, W=0.04, H=0.06, dp=0.002, rho0=1000.0, c0=20.0, g=9.81, eta=0.0,
                       jitter_amp=0.0):
    """Water column at rest in a walled tank (floor and both sides), free surface on top."""
    rng = np.random.default_rng(seed)
    fr = lattice((0.0, 0.0), (W, H), dp)
    fr = jitter(fr, dp, jitter_amp, rng)
    wr, wn = _box_walls_2d((0.0, 0.0), (W, H + 6 * dp), dp, 4)
    p = rho0 * g * (H - fr[:, 1])
    return Case(
        name="hydrostatic", dim=2, gravity=(0.0, -g, 0.0), free_surface=1, n_reinit=4,
        domain_lo=(-5 * dp, -5 * dp, 0.0), domain_hi=(W + 5 * dp, H + 12 * dp, 0.0),
        f_r=fr, f_v=np.zeros_like(fr), f_p=p, f_dp=dp, f_rho0=rho0, f_c0=c0, f_eta=eta,
        w_r=wr, w_n=wn, w_dp=dp,
        s_r0=_empty(2), s_v0=_empty(2), s_n0=_empty(2), s_cons=np.zeros(0, np.uint8),
        s_dp=dp / 2, s_rho0=1.0, s_E=1.0, s_nu=0.3,
    )


def cantilever(L=0.35, t=0.02, dpS=0.005, rho=10.0, E=1.4e3, nu=0.4, v_tip=0.05, clamp_len=None):
    """Solid-only clamped beam (2-D plane strain) for the first bending mode.

    The beam occupies x in [0, L] (free part) plus a clamp of 4 constrained
    columns at x < 0; an initial transverse velocity v_y = v_tip (x/L)^2 excites
    mostly the first mode.
    """
    clamp = 4 * dpS if clamp_len is None else clamp_len
    sr = lattice((-clamp, 0.0), (L, t), dpS)
    cons = (sr[:, 0] < 0.0).astype(np.uint8)
    sv = np.zeros_like(sr)
    sv[:, 1] = v_tip * np.clip(sr[:, 0] / L, 0.0, None) ** 2
    sn = _rect_normals(sr, -clamp, L, 0.0, t)
    tip = int(np.argmin((sr[:, 0] - (L - dpS / 2)) ** 2 + (sr[:, 1] - (t / 2 - dpS / 2)) ** 2))
    return Case(
        name="cantilever", dim=2, gravity=(0.0, 0.0, 0.0),
        domain_lo=(-0.1, -0.3, 0.0), domain_hi=(L + 0.1, 0.3, 0.0),
        f_r=_empty(2), f_v=_empty(2), f_p=np.zeros(0), f_dp=2 * dpS, f_rho0=1.0, f_c0=1.0,
        w_r=_empty(2), w_n=_empty(2), w_dp=2 * dpS,
        s_r0=sr, s_v0=sv, s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=rho, s_E=E, s_nu=nu,
        tip=tip, meta=dict(L=L, t=t),
    )


# --------------------------------------------------------------------------
# Paper benchmarks at the workload sizes
# --------------------------------------------------------------------------

def channel_flag(seed=0, D=0.1, dpF=None, ratio=2, jitter_amp=1e-3, t_ramp=0.0, L_D=25.0, H_D=4.1,
                 flag_len=3.5, flag_thick=0.2, rho_S=10.0, E=1.4e3, nu=0.4, cy_D=2.0):
    """2-D channel flow past a rigid cylinder carrying an elastic flag (Section 4.1).

    Channel 25D x 4.1D, periodic in x with a velocity-imposing inflow buffer of
    width 4 dp_F; cylinder (diameter D) centred at (2D, 2D); flag 3.5D long and
    0.2D thick attached to the cylinder's downstream side on its centre line.
    rho_F = 1, nu = 1e-3 (Re = 100), U_mean = 1, c0 = 10 U_max = 15;
    rho_S = 10, E = 1.4e3, Poisson 0.4; fluid spacing D/10, solid spacing D/20.
    Solid particles inside the cylinder are constrained (rigid).
    The initial fluid velocity is the inflow profile everywhere; with an
    inflow ramp (t_ramp > 0, Section 4.1: t_s = 2 D/U) the fluid starts at rest.

    L_D x H_D (channel size in D), cy_D (cylinder centre height in D),
    flag_len and flag_thick (in D), rho_S, E and nu override those values for
    the batched variants (flag_batch).
    """
    rng = np.random.default_rng(seed)
    dpF = D / 10 if dpF is None else dpF
    dpS = dpF / ratio
    Lx, H = L_D * D, H_D * D
    cx, cy, R = 2 * D, cy_D * D, D / 2
    fx1 = cx + R + flag_len * D
    fy0, fy1 = cy - 0.5 * flag_thick * D, cy + 0.5 * flag_thick * D

    def in_body(p):
        inc = (p[:, 0] - cx) ** 2 + (p[:, 1] - cy) ** 2 < R * R
        inf = (p[:, 0] > cx) & (p[:, 0] < fx1) & (p[:, 1] > fy0) & (p[:, 1] < fy1)
        return inc | inf, inc

    fr = lattice((0.0, 0.0), (Lx, H), dpF)
    body, _ = in_body(fr)
    fr = fr[~body]
    sr = lattice((cx - R - dpS, cy - R - dpS), (fx1 + dpS, cy + R + dpS), dpS)
    body, inc = in_body(sr)
    sr, inc = sr[body], inc[body]
    cons = inc.astype(np.uint8)
    # normals: radial on the cylinder, nearest flag face elsewhere
    sn = np.zeros_like(sr)
    rad = sr - np.array([cx, cy])
    rn = rad / np.maximum(np.linalg.norm(rad, axis=1), 1e-12)[:, None]
    fn = _rect_normals(sr, cx, fx1, fy0, fy1, faces=("r", "b", "t"))
    sn[:] = np.where(inc[:, None], rn, fn)
    wr_b, wn_b = _wall_layers_y(0.0, Lx, 0.0, -1, dpF, 4, 2)
    wr_t, wn_t = _wall_layers_y(0.0, Lx, H, +1, dpF, 4, 2)
    wr, wn = np.concatenate([wr_b, wr_t]), np.concatenate([wn_b, wn_t])
    fr = jitter(fr, dpF, jitter_amp, rng)
    sr = jitter(sr, dpS, jitter_amp, rng)
    fr[:, 0] = np.mod(fr[:, 0], Lx)
    U = 1.0
    fv = np.zeros_like(fr)
    yy = np.clip(fr[:, 1], 0.0, H)
    if t_ramp <= 0.0:
        fv[:, 0] = 6.0 * U * yy * (H - yy) / (H * H)   # parabolic inflow profile (mean U)
    # observer: free-end particle on the flag centre line
    tip_c = np.where(cons == 0)[0]
    tip = int(tip_c[np.argmin((sr[tip_c, 0] - fx1) ** 2 + (sr[tip_c, 1] - cy) ** 2)])
    c0 = 10 * 1.5 * U
    return Case(
        name="channel_flag", dim=2, gravity=(0.0, 0.0, 0.0),
        periodic_x=1, x_lo=0.0, Lx=Lx, n_reinit=5,
        inflow_on=1, inflow_profile=0, inflow_width=4 * dpF, inflow_y0=0.0, inflow_H=H,
        inflow_U=U, inflow_tramp=t_ramp,
        domain_lo=(0.0, -6 * dpF, 0.0), domain_hi=(Lx, H + 6 * dpF, 0.0),
        f_r=fr, f_v=fv, f_p=np.zeros(len(fr)), f_dp=dpF, f_rho0=1.0, f_c0=c0, f_eta=1e-3,
        w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=np.zeros_like(sr), s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=rho_S,
        s_E=E, s_nu=nu, tip=tip, meta=dict(D=D),
    )


def flag_batch(seed=0, n=256, nf_lo=2000, nf_hi=60000, D=0.1, jitter_amp=1e-3):
    """Many independent cylinder-plus-flag channels of uneven size (batched workload).

    Per instance b (own generator seeded from (seed, b)): a target fluid count
    log-uniform in [nf_lo, nf_hi]; flag length uniform in [2D, 4D], thickness
    uniform in [0.1D, 0.3D]; E log-uniform in [5e2, 5e4]; rho_S / rho_F
    uniform in [1, 20]; the discretisation of channel_flag (dp_F = D/10,
    dp_S = D/20).  The channel area is the target count times dp_F^2 plus the
    body; the height is 4.1D scaled like the square root of that area (at
    least 2.5D) and the length the rest (at least the flag's end + 2D).
    Returns a list of Case.
    """
    dpF = D / 10
    out = []
    for b in range(n):
        rng = np.random.default_rng([seed, b])
        nf = math.exp(rng.uniform(math.log(nf_lo), math.log(nf_hi)))
        fl = rng.uniform(2.0, 4.0)
        ft = rng.uniform(0.1, 0.3)
        E = math.exp(rng.uniform(math.log(5e2), math.log(5e4)))
        rho_S = rng.uniform(1.0, 20.0)
        area = nf * dpF * dpF / (D * D) + math.pi / 4 + fl * ft   # in D^2
        H_D = max(2.5, 4.1 * math.sqrt(area / (25.0 * 4.1)))
        L_D = max(area / H_D, 2.5 + fl + 2.0)
        # whole numbers of fluid spacings in both directions
        H_D = round(H_D * 10) / 10
        L_D = round(L_D * 10) / 10
        c = channel_flag(seed=int(rng.integers(1 << 30)), D=D, dpF=dpF, jitter_amp=jitter_amp, L_D=L_D,
                         H_D=H_D, flag_len=fl, flag_thick=ft, rho_S=rho_S, E=E, cy_D=H_D / 2)
        c.name = f"flag_batch[{b}]"
        c.meta.update(L_D=L_D, H_D=H_D, flag_len=fl, flag_thick=ft)
        out.append(c)
    return out


def dam_gate(seed=0, dpF=1e-3, ratio=2, jitter_amp=1e-3, E=12e6, tank_len=0.5):
    """2-D dam break through an elastic rubber gate (Section 4.2).

    Water column 0.1 m wide x 0.14 m high (rho = 1000, c0 = 20, inviscid,
    hydrostatic initial pressure) on the left of a tank of length tank_len with
    a floor and side walls; rubber gate 0.079 m free length x 0.005 m thick at
    the column's right face, its tip 1 dp_F above the floor, clamped by four
    rows of constrained particles above its free length; a rigid wall above the
    clamp closes the column.  rho_S = 1100, E = 12 MPa, Poisson 0.47.
    """
    rng = np.random.default_rng(seed)
    dpS = dpF / ratio
    Wc, Hc = 0.1, 0.14
    gx0, gx1 = Wc, Wc + 0.005
    gy0 = dpF
    gy1 = gy0 + 0.079
    clamp_h = 4 * dpS
    fr = lattice((0.0, 0.0), (Wc, Hc), dpF)
    sr = lattice((gx0, gy0), (gx1, gy1 + clamp_h), dpS)
    cons = (sr[:, 1] > gy1).astype(np.uint8)
    sn = _rect_normals(sr, gx0, gx1, gy0, gy1 + clamp_h, faces=("l", "r", "b"))
    wr, wn = _box_walls_2d((0.0, 0.0), (tank_len, 0.2), dpF, 4)
    # rigid wall closing the column above the clamp
    top0 = gy1 + clamp_h
    rw = lattice((gx0, top0), (gx1, 0.2), dpF)
    rn = _rect_normals(rw, gx0, gx1, top0, 0.2, faces=("l", "r", "b"))
    wr, wn = np.concatenate([wr, rw]), np.concatenate([wn, rn])
    fr = jitter(fr, dpF, jitter_amp, rng)
    sr = jitter(sr, dpS, jitter_amp, rng)
    p = 1000.0 * 9.81 * (Hc - fr[:, 1])
    free = np.where(cons == 0)[0]
    tip = int(free[np.argmin((sr[free, 1] - gy0) ** 2 + 1e-3 * (sr[free, 0] - gx1) ** 2)])
    return Case(
        name="dam_gate", dim=2, gravity=(0.0, -9.81, 0.0), free_surface=1, n_reinit=4,
        domain_lo=(-6 * dpF, -6 * dpF, 0.0), domain_hi=(tank_len + 6 * dpF, 0.3, 0.0),
        f_r=fr, f_v=np.zeros_like(fr), f_p=p, f_dp=dpF, f_rho0=1000.0, f_c0=20.0, f_eta=0.0,
        w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=np.zeros_like(sr), s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=1100.0,
        s_E=E, s_nu=0.47, tip=tip,
    )


def venous_valve(seed=0, wo=10.0, DH=4e-3, L_H=8.0, leaflet_H=0.4, angle_deg=60.0, b=0.2e-3, ratio=2,
                 jitter_amp=1e-3, A=2500.0, T=0.6):
    """2-D vein with two straight flexible leaflets under a pulsatile inflow
    (Section 4.3, Appendix A).

    Printed: leaflet thickness b = 0.2 mm, dp_S = b/4, dp_F = 2 dp_S; blood
    rho_F = 1000, leaflets rho_S = 1060, E = 1.5 MPa, Poisson 0.49
    (neo-Hookean); inflow driven by dp/dx = -A cos(2 pi t / T) with
    A = 2500 N/m^3, T = 0.6 s; Wo = (H/2) sqrt(omega / nu) in {1, 5, 10}, the
    viscosity following from Wo.  The geometry is in a figure that is not in
    the text; read as: channel height DH = 4 mm and length L_H DH, periodic in
    x with the Womersley profile imposed in a 4 dp_F inflow buffer; one
    leaflet rooted on each wall at x = 0.3 L, length leaflet_H DH, inclined
    downstream at angle_deg to its wall, its part inside the wall (4 dp_S)
    clamped.  c0 = 30 (A / (rho omega)) min(1, Wo^2 / 2): ten times three
    times the inflow's velocity scale (Poiseuille amplitude at small Wo, plug
    amplitude at large Wo; three for the acceleration through the gap).  The
    initial fluid velocity is zero; the observer is the top leaflet's tip.
    """
    rng = np.random.default_rng(seed)
    dpS = b / 4.0
    dpF = ratio * dpS
    L, H = L_H * DH, DH
    w = 2.0 * np.pi / T
    rho_F = 1000.0
    nu = w * (H / 2) ** 2 / wo ** 2
    c0 = 30.0 * A / (rho_F * w) * min(1.0, wo * wo / 2.0)
    th = np.radians(angle_deg)
    ll = leaflet_H * DH
    xr = 0.3 * L
    c_in = 4 * dpS
    nx_, ne_ = int(round((ll + c_in) / dpS)), int(round(b / dpS))
    xi = -c_in + (np.arange(nx_) + 0.5) * dpS
    eta = -b / 2 + (np.arange(ne_) + 0.5) * dpS
    XI, ETA = [g.ravel() for g in np.meshgrid(xi, eta, indexing="ij")]
    srs, sns, scs, stips = [], [], [], []
    leaflets = []
    for root_y, sgn in ((0.0, 1.0), (H, -1.0)):
        a = np.array([np.cos(th), sgn * np.sin(th)])
        n = np.array([-a[1], a[0]])
        root = np.array([xr, root_y])
        leaflets.append((root, a, n))
        r = root + XI[:, None] * a + ETA[:, None] * n
        # outward normal of the nearest face: the two long sides and the tip
        d_side = b / 2 - np.abs(ETA)
        d_tip = ll - XI
        nrm = np.where((d_tip < d_side)[:, None], a, np.sign(ETA)[:, None] * n)
        srs.append(r)
        sns.append(nrm)
        scs.append((XI < 0.0).astype(np.uint8))
        stips.append(np.argmin((XI - XI.max()) ** 2 + ETA ** 2 * 1e-3))
    sr = np.concatenate(srs)
    sn = np.concatenate(sns)
    cons = np.concatenate(scs)
    tip = len(srs[0]) + int(stips[1])   # the top leaflet's free end
    fr = lattice((0.0, 0.0), (L, H), dpF)
    keep = np.ones(len(fr), bool)
    for root, a, n in leaflets:
        q = fr - root
        xi_f, eta_f = q @ a, q @ n
        keep &= ~((xi_f > -c_in) & (xi_f < ll + 0.25 * dpF) & (np.abs(eta_f) < b / 2 + 0.25 * dpF))
    fr = fr[keep]
    wr_b, wn_b = _wall_layers_y(0.0, L, 0.0, -1, dpF, 4, 2)
    wr_t, wn_t = _wall_layers_y(0.0, L, H, +1, dpF, 4, 2)
    wr, wn = np.concatenate([wr_b, wr_t]), np.concatenate([wn_b, wn_t])
    fr = jitter(fr, dpF, jitter_amp, rng)
    sr = jitter(sr, dpS, jitter_amp, rng)
    fr[:, 0] = np.mod(fr[:, 0], L)
    return Case(
        name=f"venous_valve_wo{wo:g}", dim=2, gravity=(0.0, 0.0, 0.0),
        periodic_x=1, x_lo=0.0, Lx=L, n_reinit=5,
        inflow_on=1, inflow_profile=2, inflow_width=4 * dpF, inflow_y0=0.0, inflow_H=H,
        inflow_U=A / rho_F, inflow_tramp=0.0, inflow_period=T, inflow_wo=wo,
        domain_lo=(0.0, -6 * dpF, 0.0), domain_hi=(L, H + 6 * dpF, 0.0),
        f_r=fr, f_v=np.zeros_like(fr), f_p=np.zeros(len(fr)), f_dp=dpF, f_rho0=rho_F, f_c0=c0,
        f_eta=rho_F * nu, w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=np.zeros_like(sr), s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=1060.0,
        s_E=1.5e6, s_nu=0.49, tip=tip, meta=dict(DH=DH, L=L, T=T, wo=wo),
    )


def duct_plate_3d(seed=0, scale=1, jitter_amp=1e-3):
    """3-D channel flow past a clamped flexible plate.

    Duct 6 x 2 x 2 (periodic in x, walls on y and z), inflow of mean 1
    through a 4 dp_F buffer with the duct profile (parabolic across y and
    across z, zero on the four walls; a uniform plug against the no-slip
    walls ran away at the buffer's corners within 0.2-0.9 s in every setting
    tried), the fluid starting with that profile, density reinitialisation
    every 3 steps; plate 1.0 high x 0.4 span x 0.02 thick normal to the
    flow, centred 1.5 downstream of the inlet and clamped at the duct floor
    by 2 rows of constrained particles; rho_S/rho_F = 10, E = 1e4, Poisson
    0.45, nu = 0.01 (Re = 100 on the plate height and the mean velocity),
    c0 = 15.  scale=1: dp_F = 0.02, dp_S = 0.005; scale=2 doubles both
    spacings (the 1/8-size copy).
    """
    rng = np.random.default_rng(seed)
    dpF = 0.02 * scale
    dpS = 0.005 * scale
    L = (6.0, 2.0, 2.0)
    fr = lattice((0, 0, 0), L, dpF)
    p_lo = (1.5 - 0.01, 0.0, 1.0 - 0.2)
    p_hi = (1.5 + 0.01, 1.0, 1.0 + 0.2)
    clamp = 2 * dpS
    sr = lattice((p_lo[0], -clamp, p_lo[2]), p_hi, dpS)
    cons = (sr[:, 1] < 0.0).astype(np.uint8)
    # fluid displaced by the plate
    pad = np.array([0.5 * dpF, 0.0, 0.0])
    inside = np.all((fr > np.array(p_lo) - pad) & (fr < np.array(p_hi) + pad), axis=1)
    fr = fr[~inside]
    dists = np.stack([sr[:, 0] - p_lo[0], p_hi[0] - sr[:, 0], p_hi[1] - sr[:, 1],
                      sr[:, 2] - p_lo[2], p_hi[2] - sr[:, 2]], 1)
    dirs = np.array([[-1, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], float)
    sn = dirs[np.argmin(dists, 1)]
    Lw = 4 * dpF
    # walls on y (floor/ceiling) and z (side walls), full length in x
    wr = lattice((0.0, -Lw, -Lw), (L[0], L[1] + Lw, L[2] + Lw), dpF)
    inside = (wr[:, 1] > 0) & (wr[:, 1] < L[1]) & (wr[:, 2] > 0) & (wr[:, 2] < L[2])
    wr = wr[~inside]
    wn = np.zeros_like(wr)
    wn[:, 1] = np.where(wr[:, 1] < 0, 1.0, np.where(wr[:, 1] > L[1], -1.0, 0.0))
    wn[:, 2] = np.where(wr[:, 2] < 0, 1.0, np.where(wr[:, 2] > L[2], -1.0, 0.0))
    wn /= np.linalg.norm(wn, axis=1)[:, None]
    fr = jitter(fr, dpF, jitter_amp, rng)
    sr = jitter(sr, dpS, jitter_amp, rng)
    fr[:, 0] = np.mod(fr[:, 0], L[0])
    # initial velocity: the inflow profile (mean 1) at every particle's y, z
    fv = np.zeros_like(fr)
    fy = 6.0 * fr[:, 1] * (L[1] - fr[:, 1]) / L[1] ** 2
    fz = 6.0 * fr[:, 2] * (L[2] - fr[:, 2]) / L[2] ** 2
    fv[:, 0] = np.clip(fy, 0.0, None) * np.clip(fz, 0.0, None)
    free = np.where(cons == 0)[0]
    tip = int(free[np.argmax(sr[free, 1] - 1e-3 * np.abs(sr[free, 2] - 1.0))])
    return Case(
        name="duct_plate_3d", dim=3, gravity=(0.0, 0.0, 0.0), periodic_x=1, x_lo=0.0, Lx=L[0],
        n_reinit=3, inflow_on=1, inflow_profile=3, inflow_width=4 * dpF, inflow_y0=0.0,
        inflow_H=L[1], inflow_z0=0.0, inflow_Hz=L[2], inflow_U=1.0, inflow_tramp=0.0,
        domain_lo=(0.0, -6 * dpF, -6 * dpF), domain_hi=(L[0], L[1] + 6 * dpF, L[2] + 6 * dpF),
        f_r=fr, f_v=fv, f_p=np.zeros(len(fr)), f_dp=dpF, f_rho0=1.0, f_c0=15.0, f_eta=0.01,
        w_r=wr, w_n=wn, w_dp=dpF,
        s_r0=sr, s_v0=np.zeros_like(sr), s_n0=sn, s_cons=cons, s_dp=dpS, s_rho0=10.0,
        s_E=1e4, s_nu=0.45, tip=tip,
    )


BUILDERS = dict(tiny_box=tiny_box, tiny_box_3d=tiny_box_3d, floating_block=floating_block,
                hydrostatic=hydrostatic_column, cantilever=cantilever,
                channel_flag=channel_flag, dam_gate=dam_gate, duct_plate_3d=duct_plate_3d,
                flag_batch=flag_batch)

"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: quadrature,
finite differences of a stated energy, brute force, a library k-d tree,
closed forms (Euler-Bernoulli, plane Poiseuille, hydrostatics) and exact
conservation laws.  No GPU is used.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize, spatial

import fsi_cases as fc
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# --------------------------------------------------------------------------
# Kernel (Section 4: 5th-order Wendland, h = 1.3 dp; support 2h, reading R1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_unit_integral(dim):
    h = 0.37
    f = (lambda r: 2 * math.pi * r * O.kernel_W(2, r, h)) if dim == 2 else \
        (lambda r: 4 * math.pi * r * r * O.kernel_W(3, r, h))
    val, _ = integrate.quad(f, 0.0, 2 * h, epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_matches_finite_difference(dim):
    h = 0.013
    for q in (0.1, 0.5, 1.0, 1.37, 1.9):
        r, eps = q * h, 1e-7 * h
        fd = (O.kernel_W(dim, r + eps, h) - O.kernel_W(dim, r - eps, h)) / (2 * eps)
        assert abs(O.kernel_dW(dim, r, h) - fd) < 1e-6 * abs(fd)


def test_kernel_compact_support():
    h = 0.5
    for dim in (2, 3):
        assert O.kernel_W(dim, 2 * h, h) == 0.0 and O.kernel_dW(dim, 2 * h, h) == 0.0
        assert O.kernel_W(dim, 2 * h * (1 - 1e-9), h) < 1e-30
        assert O.kernel_dW(dim, 0.0, h) == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_partition_of_unity(dim):
    """Sum_j V_j W_ij on a lattice at h = 1.3 dp is 1 to within 1.1 % and the
    gradient sum vanishes by symmetry (Section 4, kernel choice)."""
    dp = 1.0
    s = O.lattice_sigma0(dim, dp, 1.3 * dp)
    assert abs(s - 1.0) < 0.011
    # jittered lattice, interior particle
    rng = np.random.default_rng(3)
    n = 9 if dim == 2 else 7
    pts = fc.lattice((0,) * dim, (n * dp,) * dim, dp)
    pts = fc.jitter(pts, dp, 1e-3, rng)
    c = np.argmin(((pts - n * dp / 2) ** 2).sum(1))
    tot, grad = 0.0, np.zeros(dim)
    for j in range(len(pts)):
        d = pts[c] - pts[j]
        r = math.sqrt((d * d).sum())
        tot += O.kernel_W(dim, r, 1.3) * dp ** dim
        if j != c:
            grad += O.kernel_dW(dim, r, 1.3) * d / r * dp ** dim
    assert abs(tot - 1.0) < 0.03
    assert np.abs(grad).max() < 0.05


# --------------------------------------------------------------------------
# Neighbour sets: brute force is the definition (r^2 < (2h)^2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_cell_list_equals_brute_force(dim, periodic):
    rng = np.random.default_rng(11 + dim + 7 * periodic)
    n = 1500 if dim == 2 else 1200
    L = 1.0
    A = rng.uniform(0, L, size=(n, dim))
    B = rng.uniform(0, L, size=(n // 2, dim))
    rc = 0.06 if dim == 2 else 0.12
    case = fc.Case(name="x", dim=dim, gravity=(0, 0, 0), periodic_x=periodic, x_lo=0.0, Lx=L)
    for same, X, Y in ((1, A, A), (0, A, B), (0, B, A)):
        p1, i1 = O.pairs(case, X, Y, rc, same, brute=False)
        p2, i2 = O.pairs(case, X, Y, rc, same, brute=True)
        assert np.array_equal(p1, p2) and np.array_equal(i1, i2)
    # against an independent library k-d tree
    box = [L] + [1e9] * (dim - 1) if periodic else None
    Bs = B.copy()
    tree = spatial.cKDTree(Bs, boxsize=box)
    p, i = O.pairs(case, A, B, rc, 0)
    for a in range(0, n, 37):
        ref = sorted(tree.query_ball_point(A[a], rc))
        assert list(i[p[a]:p[a + 1]]) == ref


def test_neighbor_counts_on_lattice():
    """20 neighbours in 2-D and 80 in 3-D at h = 1.3 dp, support 2h."""
    for dim, expect in ((2, 20), (3, 80)):
        n = 11 if dim == 2 else 9
        pts = fc.lattice((0,) * dim, (float(n),) * dim, 1.0)
        c = int(np.argmin(((pts - n / 2) ** 2).sum(1)))
        case = fc.Case(name="x", dim=dim, gravity=(0, 0, 0))
        p, i = O.pairs(case, pts[c:c + 1], pts, 2.6, 0)
        assert p[1] - p[0] == expect + 1  # self included when same=0


# --------------------------------------------------------------------------
# Equation of state (Eq. eqeos) and its inverse
# --------------------------------------------------------------------------

def test_eos_closed_forms():
    rho0, c0 = 1000.0, 20.0
    assert O.eos_p(rho0, rho0, c0) == 0.0
    eps = 1e-4
    dpdrho = (O.eos_p(rho0 + eps, rho0, c0) - O.eos_p(rho0 - eps, rho0, c0)) / (2 * eps)
    assert abs(dpdrho - c0 * c0) < 1e-6 * c0 * c0   # dp/drho = c^2 at rho0
    for p in (-5e3, -1.0, 0.0, 3.7, 1373.0, 1e5):
        rr = O.eos_rho(p, rho0, c0)
        assert abs(O.eos_p(rr, rho0, c0) - p) <= 1e-14 * max(abs(p), rho0 * c0 * c0 / 7)


# --------------------------------------------------------------------------
# Riemann interface (reading R4): reduces to the average for equal states,
# symmetric under exchange, dissipative in compression
# --------------------------------------------------------------------------

def test_riemann_properties():
    rng = np.random.default_rng(5)
    for dim in (2, 3):
        for _ in range(20):
            e = rng.normal(size=dim)
            e /= np.linalg.norm(e)
            v = rng.normal(size=dim)
            p = rng.uniform(-10, 10)
            ps, vs = O.riemann(e, v, v, p, p, 1.0, 1.0, 10.0)
            assert abs(ps - p) < 1e-12 and np.allclose(vs, v, atol=1e-12)
            vL, vR = rng.normal(size=dim), rng.normal(size=dim)
            pL, pR, rL, rR = rng.uniform(-5, 5), rng.uniform(-5, 5), 1.01, 0.99
            ps1, vs1 = O.riemann(e, vL, vR, pL, pR, rL, rR, 10.0)
            ps2, vs2 = O.riemann(-e, vR, vL, pR, pL, rR, rL, 10.0)
            assert abs(ps1 - ps2) < 1e-12 and np.allclose(vs1, vs2, atol=1e-12)
    # approaching particles raise the interface pressure, capped by c0
    e = np.array([1.0, 0.0])
    ps, _ = O.riemann(e, np.array([1.0, 0]), np.array([-1.0, 0]), 0.0, 0.0, 1.0, 1.0, 10.0)
    assert ps > 0
    ps_far, _ = O.riemann(e, np.array([100.0, 0]), np.array([-100.0, 0]), 0.0, 0.0, 1.0, 1.0, 10.0)
    assert abs(ps_far - 0.5 * 1.0 * 10.0 * 200.0) < 1e-9


# --------------------------------------------------------------------------
# Neo-Hookean stress (Eqs. Neo-Hookean-energy, 2rd-PK): P = dW/dF
# --------------------------------------------------------------------------

def _energy(F, mu, lam):
    """Strain energy of Eq. Neo-Hookean-energy: mu tr E - mu ln J + lam/2 (ln J)^2."""
    d = F.shape[0]
    E = 0.5 * (F.T @ F - np.eye(d))
    lnJ = math.log(np.linalg.det(F))
    return mu * np.trace(E) - mu * lnJ + 0.5 * lam * lnJ ** 2


@pytest.mark.parametrize("dim", [2, 3])
def test_neo_hookean_is_energy_derivative(dim):
    rng = np.random.default_rng(dim)
    mu, lam = 3.1, 7.3
    for _ in range(5):
        F = np.eye(dim) + 0.2 * rng.normal(size=(dim, dim))
        if np.linalg.det(F) < 0.3:
            continue
        P = O.neo_hookean_P(F, mu, lam)
        G = np.zeros_like(F)
        eps = 1e-6
        for i in range(dim):
            for j in range(dim):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += eps
                Fm[i, j] -= eps
                G[i, j] = (_energy(Fp, mu, lam) - _energy(Fm, mu, lam)) / (2 * eps)
        assert np.abs(P - G).max() < 1e-7 * (mu + lam)


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_stress_under_rigid_rotation(dim):
    """F from positions under a finite rotation equals R; P(R) = 0 (Eq. 2rd-PK)."""
    case = fc.cantilever() if dim == 2 else fc.tiny_box_3d()
    s = O.OracleSim(case)
    if dim == 2:
        th = 0.7
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    else:
        R = spatial.transform.Rotation.from_rotvec([0.3, -0.5, 0.8]).as_matrix()
    s.set_solid_positions(s.s_r0 @ R.T + 0.123)
    F = s.F_from_positions()
    assert np.abs(F - R[None]).max() < 1e-12
    P = O.neo_hookean_P(R, 1.0, 2.0)
    assert np.abs(P).max() < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_corrected_gradient_reproduces_affine_fields(dim):
    """With B0 (Eq. correctmatrix, reading R8) F = I on the reference
    configuration and F = A under r = A r0 + b, boundary particles included."""
    case = fc.cantilever() if dim == 2 else fc.tiny_box_3d()
    s = O.OracleSim(case)
    assert np.abs(s.F_from_positions() - np.eye(dim)[None]).max() < 1e-12
    rng = np.random.default_rng(1)
    A = np.eye(dim) + 0.3 * rng.normal(size=(dim, dim))
    s.set_solid_positions(s.s_r0 @ A.T + 0.5)
    assert np.abs(s.F_from_positions() - A[None]).max() < 1e-11


def test_uniform_stretch_has_no_interior_force():
    """A uniform deformation gives a uniform stress: zero net force on interior particles."""
    case = fc.cantilever(L=0.1, t=0.08)
    s = O.OracleSim(case)
    F = np.array([[1.05, 0.02], [0.0, 0.97]])
    acc = s.solid_accel(np.broadcast_to(F, s.s_F.shape).copy())
    r = s.s_r0
    m = 4 * 1.3 * case.s_dp   # the particle and all its neighbours have full support
    interior = (r[:, 0] > -0.02 + m) & (r[:, 0] < 0.1 - m) & (r[:, 1] > m) & (r[:, 1] < 0.08 - m)
    assert interior.sum() > 10
    assert np.abs(acc[interior]).max() < 1e-8 * np.abs(acc).max()


# --------------------------------------------------------------------------
# Solid dynamics: dF/dt integration and a cantilever against Euler-Bernoulli
# --------------------------------------------------------------------------

def test_integrated_F_matches_F_from_positions():
    """Integrating dF/dt (reading R9) keeps F equal to the position-based F."""
    case = fc.cantilever(L=0.2, v_tip=0.2)
    s = O.OracleSim(case)
    _, _, dts = s.suggest_dt()
    for _ in range(100):
        s.step(5 * dts * 0.9, 5)
    F = s.F_from_positions()
    assert np.abs(F - s.s_F).max() < 1e-11
    assert np.abs(s.s_F - np.eye(2)).max() > 1e-4   # it did deform


def _cantilever_period(dpS, L=0.2):
    case = fc.cantilever(L=L, dpS=dpS, v_tip=0.02)
    s = O.OracleSim(case)
    _, _, dts = s.suggest_dt()
    dt = 0.9 * dts
    ys, ts = [], []
    while True:
        s.step(dt, 1)
        ys.append(s.s_r[case.tip, 1] - s.s_r0[case.tip, 1])
        ts.append(s.t)
        y = np.array(ys)
        down = np.where((y[:-1] > 0) & (y[1:] <= 0))[0]
        up = np.where((y[:-1] < 0) & (y[1:] >= 0))[0]
        if len(up) >= 1 and len(down) >= 1:
            # linear interpolation of the crossings
            def cross(k):
                return ts[k] + (ts[k + 1] - ts[k]) * y[k] / (y[k] - y[k + 1])
            return 2.0 * (cross(up[0]) - cross(down[0]))


def test_cantilever_first_mode_vs_euler_bernoulli():
    """Clamped 2-D plane-strain beam (L = 0.2, t = 0.02, rho = 10, E = 1.4e3,
    nu = 0.4): the period converges at second order to the Euler-Bernoulli
    value; the Richardson extrapolation of 4 and 8 layers is within 5 %."""
    g = _golden("euler_bernoulli.txt")
    b1 = optimize.brentq(lambda x: 1 + math.cos(x) * math.cosh(x), 1.0, 3.0, xtol=1e-15)
    assert abs(b1 - g["beta1L"]) < 1e-12
    L, t, E, nu, rho = 0.2, 0.02, 1.4e3, 0.4, 10.0
    Ep = E / (1 - nu * nu)
    f1 = b1 ** 2 / (2 * math.pi) * math.sqrt(Ep * t ** 3 / 12 / (rho * t * L ** 4))
    T_eb = 1 / f1
    T4 = _cantilever_period(0.005)
    T8 = _cantilever_period(0.0025)
    assert abs(T8 - T_eb) < abs(T4 - T_eb) / 2.5        # converging
    T_ext = T8 + (T8 - T4) / 3.0
    assert abs(T_ext / T_eb - 1.0) < 0.05


# --------------------------------------------------------------------------
# Coupling and integrator: antisymmetry and momentum conservation
# --------------------------------------------------------------------------

def test_fluid_solid_forces_are_antisymmetric():
    """Sum_i f_i^S + Sum_a f_a^F = 0 (Eqs. S:p, S:v vs F:p, F:v)."""
    s = O.OracleSim(fc.tiny_box(seed=2))
    dt, _, dts = s.suggest_dt()
    for _ in range(3):
        d = s.step(dt, 3)
        tot = d["mom_fs_fluid"] + d["mom_fs_solid"]
        assert d["n_fs"] > 0 and d["n_fs"] == d["n_sf"]
        assert np.abs(tot).max() <= 1e-13 * d["abs_fs"]


def test_total_momentum_conserved_with_substeps():
    """Free block in a periodic fluid blob, no walls, no gravity, K = 3:
    position-based Verlet with sum of dt_S = dt_F conserves the total momentum
    to round-off (Section 3.3)."""
    case = fc.floating_block(seed=1)
    s = O.OracleSim(case)
    mF, mS = case.f_rho0 * case.f_dp ** 2, case.s_rho0 * case.s_dp ** 2

    def mom():
        return mF * s.f_v.sum(0) + mS * s.s_v.sum(0)

    scale = mF * np.abs(s.f_v).sum() + mS * np.abs(s.s_v).sum()
    P0 = mom()
    dt, _, _ = s.suggest_dt()
    for _ in range(100):
        s.step(dt, 3)
    assert np.abs(mom() - P0).max() < 1e-13 * scale
    assert np.abs(s.s_v).max() > 1e-3   # the block moved


def test_time_averages_are_trajectory_means():
    """v~ dt_F = r^{n+1} - r^n and a~ dt_F = v^{n+1} - v^n (reading R14)."""
    s = O.OracleSim(fc.tiny_box(seed=4))
    dt, _, _ = s.suggest_dt()
    s.step(dt, 2)
    r0, v0 = s.s_r.copy(), s.s_v.copy()
    s.step(dt, 4)
    assert np.abs(s.s_vbar * dt - (s.s_r - r0)).max() < 1e-15
    assert np.abs(s.s_abar * dt - (s.s_v - v0)).max() < 1e-14


# --------------------------------------------------------------------------
# Ghost state (reading R6): hydrostatic equilibrium and no-slip Poiseuille
# --------------------------------------------------------------------------

def test_hydrostatic_column_in_equilibrium_at_the_floor():
    """A water column with hydrostatic density at rest: the near-floor fluid
    is in equilibrium only if the ghost pressure adds rho g d (reading R6)."""
    case = fc.hydrostatic_column(W=0.04, H=0.06, dp=0.002)
    case.n_reinit = 0
    s = O.OracleSim(case)
    s.step(1e-12, 1)
    a, x, y = s.f_dvdt, s.f_r[:, 0], s.f_r[:, 1]
    hF, g = 1.3 * 0.002, 9.81
    cols = (x > 2 * hF) & (x < 0.04 - 2 * hF)
    bottom = cols & (y < 2 * hF)
    interior = cols & (y > 2 * hF) & (y < 0.06 - 3 * hF)
    assert abs(a[bottom, 1].mean()) < 0.06 * g
    assert np.abs(a[interior, 1]).max() < 0.05 * g


def _poiseuille_case(steps):
    dp, H, Lx, nu, Umax = 0.001, 0.02, 0.02, 1e-3, 0.05
    g = 8 * nu * Umax / H ** 2
    fr = fc.lattice((0, 0), (Lx, H), dp)
    wb, nb = fc._wall_layers_y(0, Lx, 0.0, -1, dp, 4, 2)
    wt, nt = fc._wall_layers_y(0, Lx, H, +1, dp, 4, 2)
    case = fc.Case(name="poiseuille", dim=2, gravity=(g, 0, 0), periodic_x=1, x_lo=0, Lx=Lx,
                   f_r=fr, f_v=np.zeros_like(fr), f_p=np.zeros(len(fr)), f_dp=dp, f_rho0=1.0,
                   f_c0=2.0, f_eta=nu, w_r=np.concatenate([wb, wt]), w_n=np.concatenate([nb, nt]),
                   w_dp=dp, s_r0=np.zeros((0, 2)), s_v0=np.zeros((0, 2)), s_n0=np.zeros((0, 2)),
                   s_cons=np.zeros(0, np.uint8), s_dp=dp / 2)
    s = O.OracleSim(case)
    dt, _, _ = s.suggest_dt(vmax_f=Umax)
    for _ in range(steps):
        s.step(dt, 1)
    return s, g, nu, H, Umax


def test_plane_poiseuille_no_slip():
    """Body-force driven flow between walls reaches the parabola
    u = g y (H - y) / (2 nu) (ghost velocity 2 v~ - v_i, reading R6)."""
    s, g, nu, H, Umax = _poiseuille_case(1000)
    y, u = s.f_r[:, 1], s.f_v[:, 0]
    rows = np.round(y / 0.001 - 0.5).astype(int)
    for k in np.unique(rows):
        sel = rows == k
        ue = g * y[sel].mean() * (H - y[sel].mean()) / (2 * nu)
        assert abs(u[sel].mean() - ue) < 0.025 * Umax
    assert np.abs(s.f_v[:, 1]).max() < 1e-2 * Umax


# --------------------------------------------------------------------------
# Density reinitialisation (reading R16) and inflow (reading R18)
# --------------------------------------------------------------------------

def test_density_reinit_recovers_rho0_on_lattice():
    case = fc.hydrostatic_column(W=0.04, H=0.04, dp=0.002)
    case.f_p[:] = 0.0
    case.f_v[:] = 0.0
    case.gravity = (0.0, 0.0, 0.0)
    case.free_surface = 0
    case.n_reinit = 1
    s = O.OracleSim(case)
    s.f_rho[:] = 1234.0
    s.step(1e-12, 1)
    x, y = s.f_r[:, 0], s.f_r[:, 1]
    hF = 1.3 * 0.002
    inner = (x > 2 * hF) & (x < 0.04 - 2 * hF) & (y > 2 * hF) & (y < 0.04 - 2 * hF)
    assert np.abs(s.f_rho[inner] / 1000.0 - 1.0).max() < 1e-9
    # at the walls the wall particles complete the support
    near = (x < 2 * hF) & (y > 2 * hF) & (y < 0.04 - 2 * hF)
    assert np.abs(s.f_rho[near] / 1000.0 - 1.0).max() < 1e-9


def test_inflow_profile_mean_and_ramp():
    case = fc.channel_flag()
    P = O.make_params(case)
    H = case.inflow_H
    mean, _ = integrate.quad(lambda y: O.lib().or_inflow_u(P, y, 10.0), 0.0, H)
    assert abs(mean / H - 1.0) < 1e-12
    assert abs(O.lib().or_inflow_u(P, H / 2, 10.0) - 1.5) < 1e-12
    P.inflow_tramp = 2.0
    assert abs(O.lib().or_inflow_u(P, H / 2, 1.0) - 0.75) < 1e-12   # half-way up the ramp
    assert O.lib().or_inflow_u(P, H / 2, 0.0) == 0.0


# --------------------------------------------------------------------------
# Single-time-step baselines (Section 2.2 criterion; Section 3.2 alternative)
# --------------------------------------------------------------------------

def _dt_case(dpF=0.01, c0=10.0, eta=0.0, rho0=1.0, E=1e-6, rhoS=10.0):
    import dataclasses
    c = fc.tiny_box(seed=0, nx=8, ny=6, dpF=dpF, ratio=2, c0=c0, eta=eta, rho0=rho0)
    return O.OracleSim(dataclasses.replace(c, s_E=E, s_rho0=rhoS))


def test_single_dt_regimes_scale_as_their_physics():
    """Each term of the single-step criterion, isolated by the parameters,
    scales as its physics: the acoustic terms linearly with the particle
    spacing and inversely with the signal speed, the viscous term with the
    spacing squared over the kinematic viscosity, the acceleration term with
    the square root of spacing over acceleration."""
    def dt(mode=1, vf=0.0, vs=0.0, a=0.0, **kw):
        return _dt_case(**kw).single_dt(mode, vf, vs, a)

    # fluid acoustic (soft solid, no viscosity): 0.25 h_F / c_F at rest
    base = dt()
    assert base == pytest.approx(0.25 * 1.3 * 0.01 / 10.0, rel=1e-14)
    assert dt(dpF=0.02) == pytest.approx(2.0 * base, rel=1e-14)
    assert dt(c0=20.0) == pytest.approx(0.5 * base, rel=1e-14)
    # the largest speed of either phase adds to the sound speed
    assert dt(vf=10.0) == pytest.approx(0.5 * base, rel=1e-14)
    assert dt(vs=10.0) == pytest.approx(0.5 * base, rel=1e-14)
    # viscous: h_F^2 / nu, nu = eta / rho0
    v1 = dt(eta=1.0)
    assert v1 < base
    assert dt(eta=1.0, dpF=0.02) == pytest.approx(4.0 * v1, rel=1e-14)
    assert dt(eta=2.0) == pytest.approx(0.5 * v1, rel=1e-14)
    assert dt(eta=1.0, rho0=2.0) == pytest.approx(2.0 * v1, rel=1e-14)
    # solid acoustic (slow fluid, stiff solid): 0.6 h_S / c_S, c_S ~ sqrt(E / rho_S)
    s1 = dt(c0=1e-3, E=1e4)
    assert dt(c0=1e-3, E=4e4) == pytest.approx(0.5 * s1, rel=1e-12)
    assert dt(c0=1e-3, E=1e4, rhoS=40.0) == pytest.approx(2.0 * s1, rel=1e-12)
    assert dt(c0=1e-3, E=1e4, dpF=0.02) == pytest.approx(2.0 * s1, rel=1e-12)
    # solid acceleration: 0.6 sqrt(h_S / |dv/dt|)
    a1 = dt(c0=1e-3, E=1e-6, a=1e6)
    assert a1 == pytest.approx(0.6 * math.sqrt(1.3 * 0.005 / 1e6), rel=1e-14)
    assert dt(c0=1e-3, E=1e-6, a=4e6) == pytest.approx(0.5 * a1, rel=1e-14)
    assert dt(c0=1e-3, E=1e-6, a=1e6, dpF=0.04) == pytest.approx(2.0 * a1, rel=1e-14)


def test_single_dt_modes_bound_and_reduce():
    """The Section 2.2 step never exceeds the solid step used as a single
    step (mode 2), which is the smaller of the acoustic fluid step and the
    solid step; a fluid without a body has no solid terms."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        s = _dt_case(c0=float(rng.uniform(1, 50)), eta=float(rng.choice([0.0, 1e-3, 1.0])),
                     E=float(10 ** rng.uniform(-2, 6)))
        vf, vs, a = (float(rng.uniform(0, 5)), float(rng.uniform(0, 5)), float(10 ** rng.uniform(-3, 6)))
        m1, m2 = s.single_dt(1, vf, vs, a), s.single_dt(2, vf, vs, a)
        ac, _, dS = s.suggest_dt(vf, vs, a)
        assert m2 == min(ac, dS)
        assert m1 <= m2
        # with K = 1 the sub-step rule gives one sub-step for this step
        assert s.substeps(m2, dS) == (1 if m2 < dS else 2)
    c = fc.tiny_box(seed=0, nx=8, ny=6, with_solid=False)
    s = O.OracleSim(c)
    assert s.single_dt(1, 0.0, 0.0, 0.0) == pytest.approx(0.25 * 1.3 * c.f_dp / c.f_c0, rel=1e-14)
    assert s.single_dt(2, 0.0, 0.0, 0.0) == pytest.approx(0.6 * 1.3 * c.f_dp / c.f_c0, rel=1e-14)


# --------------------------------------------------------------------------
# Coincident particles (reading R23): the pair rule at r = 0 is the limit r -> 0+
# --------------------------------------------------------------------------

def _with_coincident(eps):
    """tiny_box plus a copy of one fluid particle and a fluid particle on a
    solid particle, each displaced by eps dp (eps = 0: on top)."""
    c = fc.tiny_box(seed=11)
    k, m = len(c.f_r) // 3, len(c.s_r0) // 2
    off = eps * c.f_dp * np.array([0.6, 0.8])
    c.f_r = np.concatenate([c.f_r, c.f_r[k:k + 1] + off, c.s_r0[m:m + 1] + off])
    c.f_v = np.concatenate([c.f_v, c.f_v[k:k + 1], c.s_v0[m:m + 1]])
    c.f_p = np.concatenate([c.f_p, c.f_p[k:k + 1], [0.0]])
    return c


def test_coincident_pairs_are_the_limit_of_close_pairs():
    out = []
    for eps in (0.0, 1e-9):
        s = O.OracleSim(_with_coincident(eps))
        dt, _, dts = s.suggest_dt()
        s.step(dt, s.substeps(dt, dts))
        assert np.all(np.isfinite(s.f_dvdt)) and np.all(np.isfinite(s.f_drho)) and np.all(np.isfinite(s.s_fF))
        out.append((s.f_dvdt.copy(), s.f_drho.copy(), s.s_fF.copy()))
    for a, b in zip(*out):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def _dyadic(x, bits=20):
    """Round to a multiple of 2^-bits, so that half drifts by dt = 2^-12 of
    velocities that are multiples of 2^-7 are exact in FP64."""
    return np.round(np.asarray(x, np.float64) * 2.0 ** bits) / 2.0 ** bits


def _coincident_at_mid_state(eps, dt):
    """tiny_box plus two fluid particles with velocities unlike their
    partners', placed so that after the first half drift (r + dt v / 2) one
    sits exactly on fluid particle k and the other exactly on solid particle
    m (both displaced by eps dp)."""
    c = fc.tiny_box(seed=11)
    c.n_reinit = 0
    k, m = len(c.f_r) // 3, len(c.s_r0) // 2
    c.f_r, c.f_v = c.f_r.copy(), c.f_v.copy()
    c.f_r[k] = _dyadic(c.f_r[k])
    c.f_v[k] = [2.0 ** -6, -2.0 ** -7]
    dv = np.array([2.0 ** -5, -3 * 2.0 ** -7])
    s0 = c.s_r0.copy()
    s0[m] = _dyadic(s0[m])
    c.s_r0 = s0
    vs = np.array([-2.0 ** -6, 2.0 ** -5])
    off = eps * c.f_dp * np.array([0.6, 0.8])
    c.f_r = np.concatenate([c.f_r, (c.f_r[k] - 0.5 * dt * dv + off)[None], (s0[m] - 0.5 * dt * vs + off)[None]])
    c.f_v = np.concatenate([c.f_v, (c.f_v[k] + dv)[None], vs[None]])
    c.f_p = np.concatenate([c.f_p, c.f_p[k:k + 1], [0.0]])
    return c, k


def test_coincident_pair_with_unequal_velocities_drops_only_the_viscous_limit():
    """Reading R23 with v_i != v_j.  As r -> 0 the Wendland kernel gives
    (1/r) dW/dr -> -5 alpha_2 / h^2 (a closed form of the kernel of Section
    4), so the fluid-fluid viscous term 2 eta V_i V_j (v_i - v_j) (1/r) dW/dr
    has a finite limit, which the coincident pair drops; the pressure terms
    vanish with dW.  The step at r = 1e-9 dp must therefore exceed the step
    at r = 0 by exactly that limit on the pair (opposite on the partner) and
    by nothing elsewhere; the fluid-solid viscous term, regularised by
    r + 0.01 h_F, has limit zero, so the particle on the solid and the solid's
    coupling force do not change."""
    dt = 2.0 ** -12
    out = []
    for eps in (0.0, 1e-9):
        case, k = _coincident_at_mid_state(eps, dt)
        s = O.OracleSim(case)
        rho = s.f_rho.copy()
        s.step(dt, 2)
        assert np.all(np.isfinite(s.f_dvdt)) and np.all(np.isfinite(s.s_fF))
        out.append((s.f_dvdt.copy(), s.s_fF.copy()))
    d = out[1][0] - out[0][0]
    i, j = k, case.nf - 2
    hF = 1.3 * case.f_dp
    alpha = 7.0 / (4.0 * math.pi * hF ** 2)
    m = case.f_rho0 * case.f_dp ** 2
    lim = 2 * case.f_eta * (m / rho[i]) * (m / rho[j]) * (case.f_v[i] - case.f_v[j]) * (-5 * alpha / hF ** 2) / m
    assert np.abs(lim).max() > 0.3     # the limit is not small: ~6 % of g here
    assert np.abs(d[i] - lim).max() <= 1e-6 * np.abs(lim).max()
    assert np.abs(d[j] + lim).max() <= 1e-6 * np.abs(lim).max()
    rest = np.ones(case.nf, bool)
    rest[[i, j]] = False
    assert np.abs(d[rest]).max() <= 1e-6 * np.abs(lim).max()
    assert np.abs(out[1][1] - out[0][1]).max() <= 1e-6 * np.abs(out[0][1]).max()


# --------------------------------------------------------------------------
# Normal update (reading R17): n = normalize(F^-T n0) at the reinit cadence
# --------------------------------------------------------------------------

def _rotation(dim, seed):
    rng = np.random.default_rng(seed)
    if dim == 2:
        th = rng.uniform(0.3, 2.5)
        return np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return spatial.transform.Rotation.from_rotvec(rng.uniform(-1.0, 1.0, 3)).as_matrix()


def _normals_after_one_reinit_step(dim, F):
    case = fc.tiny_box(seed=3) if dim == 2 else fc.tiny_box_3d(seed=3)
    case.n_reinit = 1      # step 0 is a reinitialisation step
    s = O.OracleSim(case)
    s.s_F[:] = F
    s.step(1e-9, 1)        # the normals are set before the sub-steps move F
    return s.s_n0.copy(), s.s_nrm.copy()


@pytest.mark.parametrize("dim", [2, 3])
def test_normals_turn_with_a_rigid_rotation(dim):
    """F = R (finite rotation): the surface turns with the body, n = R n0."""
    R = _rotation(dim, seed=dim)
    n0, n = _normals_after_one_reinit_step(dim, np.broadcast_to(R, (1, dim, dim)))
    assert np.abs(n - n0 @ R.T).max() < 1e-12


def _tangents(n0):
    """Unit vectors spanning the plane normal to each row of n0."""
    if n0.shape[1] == 2:
        return [np.stack([-n0[:, 1], n0[:, 0]], 1)]
    a = np.where(np.abs(n0[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    t1 = np.cross(n0, a)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    return [t1, np.cross(n0, t1)]


@pytest.mark.parametrize("dim", [2, 3])
def test_normals_of_an_affinely_deformed_surface(dim):
    """F = A (a general affine map, det A > 0, different per particle): a
    material surface element with normal n0 and tangents t maps to the
    element spanned by A t, so the new unit normal must be orthogonal to
    every A t and point to the same side as A n0 (the map keeps the
    orientation).  Checked by geometry, not by the F^-T formula."""
    rng = np.random.default_rng(7 + dim)
    case_ns = len(fc.tiny_box(seed=3).s_r0) if dim == 2 else len(fc.tiny_box_3d(seed=3).s_r0)
    A = np.eye(dim)[None] + rng.uniform(-0.45, 0.45, size=(case_ns, dim, dim))
    assert np.all(np.linalg.det(A) > 0.05)
    n0, n = _normals_after_one_reinit_step(dim, A)
    assert np.abs(np.linalg.norm(n, axis=1) - 1.0).max() < 1e-14
    for t in _tangents(n0):
        At = np.einsum("aij,aj->ai", A, t)
        assert np.abs((n * At).sum(1)).max() < 1e-13 * np.abs(At).max()
    assert np.all((n * np.einsum("aij,aj->ai", A, n0)).sum(1) > 0.0)


# --------------------------------------------------------------------------
# Inflow buffer assignment (reading R18)
# --------------------------------------------------------------------------

def test_inflow_buffer_sets_exactly_the_particles_inside_it():
    """With dt = 0 a step leaves the velocities as the inflow buffer (a1)
    set them: every fluid particle with x in [x_lo, x_lo + width) carries
    (U(y, t), 0) -- U the profile pinned above, half-way up its ramp here --
    and every other particle keeps its velocity bit for bit.  Two particles
    sit exactly on the buffer's edges (x_lo inside, x_lo + width outside)."""
    case = fc.channel_flag(t_ramp=0.5)
    rng = np.random.default_rng(5)
    case.f_v = rng.uniform(-0.3, 0.3, size=case.f_v.shape)
    edge = np.argsort(np.abs(case.f_r[:, 0] - case.inflow_width))[:1]
    lo = np.argsort(np.abs(case.f_r[:, 0] - case.x_lo))[:1]
    case.f_r = case.f_r.copy()
    case.f_r[edge, 0] = case.x_lo + case.inflow_width
    case.f_r[lo, 0] = case.x_lo
    s = O.OracleSim(case)
    s.t = 0.25
    r0, v0 = s.f_r.copy(), s.f_v.copy()
    s.step(0.0, 1)
    inb = (r0[:, 0] >= case.x_lo) & (r0[:, 0] < case.x_lo + case.inflow_width)
    assert inb[lo].all() and not inb[edge].any() and 100 < inb.sum() < case.nf // 10
    P = O.make_params(case)
    u = np.array([O.lib().or_inflow_u(P, y, 0.25) for y in r0[inb, 1]])
    assert np.array_equal(s.f_v[inb, 0], u) and np.all(s.f_v[inb, 1] == 0.0)
    assert np.array_equal(s.f_v[~inb], v0[~inb])


def _duct_params(H=2.0, Hz=1.5, y0=0.3, z0=-0.2, U=1.0):
    c = fc.tiny_box_3d()
    P = O.make_params(c)
    P.inflow_on, P.inflow_profile, P.inflow_U, P.inflow_tramp = 1, 3, U, 0.0
    P.inflow_y0, P.inflow_H, P.inflow_z0, P.inflow_Hz = y0, H, z0, Hz
    return P


def test_duct_inflow_profile_closed_forms():
    """Reading R26 on a rectangular cross-section (H != Hz, both origins
    off zero, so a swapped axis, extent or origin fails): the mean over the
    cross-section is Ubar (2-D quadrature), the value is 0 on all four walls
    and 36/16 Ubar at the centre, it is symmetric about both mid-planes,
    separable (u(y, z) u(yc, zc) = u(y, zc) u(yc, z)), clamped outside the
    section, and follows the ramp; profiles other than 3 ignore z."""
    H, Hz, y0, z0 = 2.0, 1.5, 0.3, -0.2
    P = _duct_params(H, Hz, y0, z0, U=1.3)
    u = lambda y, z, t=10.0: O.lib().or_inflow_u3(P, y, z, t)
    mean, _ = integrate.dblquad(lambda z, y: u(y, z), y0, y0 + H, z0, z0 + Hz, epsabs=1e-13, epsrel=1e-13)
    assert abs(mean / (H * Hz) - 1.3) < 1e-12
    yc, zc = y0 + H / 2, z0 + Hz / 2
    assert abs(u(yc, zc) - 1.3 * 2.25) < 1e-12
    for y in np.linspace(y0, y0 + H, 7):   # (y0 + H) - y0 rounds: zero to round-off
        assert abs(u(y, z0)) < 1e-14 and abs(u(y, z0 + Hz)) < 1e-14
    for z in np.linspace(z0, z0 + Hz, 7):
        assert abs(u(y0, z)) < 1e-14 and abs(u(y0 + H, z)) < 1e-14
    rng = np.random.default_rng(3)
    for y, z in zip(rng.uniform(y0, y0 + H, 20), rng.uniform(z0, z0 + Hz, 20)):
        assert abs(u(y, z) - u(2 * yc - y, z)) < 1e-12 and abs(u(y, z) - u(y, 2 * zc - z)) < 1e-12
        assert abs(u(y, z) * u(yc, zc) - u(y, zc) * u(yc, z)) < 1e-12
        # across y alone: the channel profile of reading R18 (6 y (H - y) / H^2), times 1.5 at mid-z
        assert abs(u(y, zc) - 1.3 * 1.5 * 6.0 * (y - y0) * (H - (y - y0)) / H ** 2) < 1e-12
    assert u(y0 - 0.5, zc) == 0.0 and u(yc, z0 + Hz + 0.5) == 0.0
    P.inflow_tramp = 2.0
    assert abs(u(yc, zc, 1.0) - 0.5 * 1.3 * 2.25) < 1e-12
    P.inflow_profile = 0
    assert O.lib().or_inflow_u3(P, yc, 123.0, 10.0) == O.lib().or_inflow_u(P, yc, 10.0)


def test_duct_inflow_buffer_sets_exactly_the_particles_inside_it():
    """The 3-D counterpart of the buffer test above: with dt = 0, fluid
    particles with x in [x_lo, x_lo + width) carry (U(y, z, t), 0, 0) with
    the duct profile evaluated at their own y and z, every other particle
    keeps its velocity bit for bit."""
    case = fc.tiny_box_3d(seed=2)
    L = case.f_r.max(0) + 0.5 * case.f_dp
    case.inflow_on, case.inflow_profile, case.inflow_U, case.inflow_tramp = 1, 3, 0.7, 0.5
    case.inflow_width, case.x_lo = 3 * case.f_dp, 0.0
    case.inflow_y0, case.inflow_H, case.inflow_z0, case.inflow_Hz = 0.0, float(L[1]), 0.0, float(L[2])
    s = O.OracleSim(case)
    s.t = 0.25
    r0, v0 = s.f_r.copy(), s.f_v.copy()
    s.step(0.0, 1)
    inb = (r0[:, 0] >= case.x_lo) & (r0[:, 0] < case.x_lo + case.inflow_width)
    assert 20 < inb.sum() < case.nf // 2
    P = O.make_params(case)
    u = np.array([O.lib().or_inflow_u3(P, y, z, 0.25) for y, z in r0[inb, 1:3]])
    assert len(np.unique(np.round(u, 12))) > 5   # the profile varies across the buffer
    assert np.array_equal(s.f_v[inb, 0], u) and np.all(s.f_v[inb, 1:] == 0.0)
    assert np.array_equal(s.f_v[~inb], v0[~inb])


# --------------------------------------------------------------------------
# Womersley inflow (Appendix A, reading R24)
# --------------------------------------------------------------------------

def _womersley_params(wo, H=5e-3, T=0.6, A_rho=2.5):
    c = fc.channel_flag()
    P = O.make_params(c)
    P.inflow_profile, P.inflow_y0, P.inflow_H, P.inflow_U = 2, 0.0, H, A_rho
    P.inflow_period, P.inflow_wo, P.inflow_tramp = T, wo, 0.0
    w = 2 * math.pi / T
    nu = w * (H / 2) ** 2 / wo ** 2
    return P, w, nu


@pytest.mark.parametrize("wo", [1.0, 5.0, 10.0])
def test_womersley_profile_solves_the_oscillating_channel_flow(wo):
    """u(y, t) satisfies u_t = (A/rho) cos(omega t) + nu u_yy (central
    differences), vanishes on both walls and is periodic in T."""
    P, w, nu = _womersley_params(wo)
    H, U, T = P.inflow_H, P.inflow_U, P.inflow_period
    u = lambda y, t: O.lib().or_inflow_u(P, y, t)
    scale = U / w
    for t in (0.0, 0.07, 0.21, 0.44):
        assert abs(u(0.0, t)) < 1e-12 * scale and abs(u(H, t)) < 1e-12 * scale
        assert abs(u(0.3 * H, t + T) - u(0.3 * H, t)) < 1e-12 * scale
        for y in np.linspace(0.1, 0.9, 7) * H:
            et, ey = 1e-5 * T, 1e-3 * H
            ut = (u(y, t + et) - u(y, t - et)) / (2 * et)
            uyy = (u(y + ey, t) - 2 * u(y, t) + u(y - ey, t)) / ey ** 2
            res = ut - U * math.cos(w * t) - nu * uyy
            assert abs(res) < 2e-5 * U, (wo, t, y, res)


def test_womersley_low_frequency_limit_is_poiseuille():
    """Wo -> 0: the profile is the steady channel flow of the instantaneous
    pressure gradient, (A / (2 rho nu)) (y)(H - y) cos(omega t)."""
    P, w, nu = _womersley_params(0.02)
    H, U = P.inflow_H, P.inflow_U
    for t in (0.0, 0.1, 0.25):
        for y in (0.2 * H, 0.5 * H, 0.7 * H):
            want = U / (2 * nu) * y * (H - y) * math.cos(w * t)
            got = O.lib().or_inflow_u(P, y, t)
            assert abs(got - want) < 1e-3 * U / (2 * nu) * H * H / 4


# --------------------------------------------------------------------------
# Neighbour lists and kernel values held over an advection step (reading F2)
# --------------------------------------------------------------------------

def test_advection_cadence_one_is_the_per_step_rebuild():
    case = fc.tiny_box(seed=3)
    a, b = O.OracleSim(case), O.OracleSim(case)
    b.set_advection_cadence(1)
    dt, _, dts = a.suggest_dt()
    K = a.substeps(dt, dts)
    for _ in range(6):
        a.step(dt, K)
        b.step(dt, K)
    for x, y in ((a.f_r, b.f_r), (a.f_v, b.f_v), (a.f_rho, b.f_rho), (a.s_r, b.s_r), (a.s_F, b.s_F)):
        assert np.array_equal(x, y)


def test_frozen_configuration_conserves_momentum_and_its_pair_counts():
    """With the configuration held for 4 steps the pair terms still act
    through one geometry on both sides, so the free block in fluid conserves
    the total momentum to round-off; the pair counts stay those of the step
    that built the configuration."""
    case = fc.floating_block(seed=1)
    s = O.OracleSim(case)
    s.set_advection_cadence(4)
    mF, mS = case.f_rho0 * case.f_dp ** 2, case.s_rho0 * case.s_dp ** 2

    def mom():
        return mF * s.f_v.sum(0) + mS * s.s_v.sum(0)

    scale = mF * np.abs(s.f_v).sum() + mS * np.abs(s.s_v).sum()
    P0 = mom()
    dt, _, _ = s.suggest_dt()
    counts = []
    for _ in range(40):
        d = s.step(dt, 3)
        counts.append((d["n_ff"], d["n_fs"], d["n_sf"]))
    assert np.abs(mom() - P0).max() < 1e-13 * scale
    assert np.abs(s.s_v).max() > 1e-3
    for w0 in range(0, 40, 4):
        assert len(set(counts[w0:w0 + 4])) == 1
    assert len(set(counts)) > 1   # the lists were rebuilt as the flow moved


def _translating_block(U=(0.7, 0.4), eta=0.0, dp=0.01, n=10):
    """A free fluid block (no walls, body, gravity, initial pressure or
    reinitialisation) moving rigidly: no pair term acts, its speed stays |U|."""
    r = fc.lattice((0.0, 0.0), (n * dp, n * dp), dp)
    return fc.Case(name="translating_block", dim=2, gravity=(0.0, 0.0, 0.0),
                   domain_lo=(-1.0, -1.0, 0.0), domain_hi=(2.0, 2.0, 1.0),
                   f_r=r, f_v=np.tile(np.asarray(U, float), (len(r), 1)), f_p=np.zeros(len(r)), f_dp=dp,
                   f_rho0=1.0, f_c0=10.0, f_eta=eta, w_r=np.zeros((0, 2)), w_n=np.zeros((0, 2)), w_dp=dp,
                   s_r0=np.zeros((0, 2)), s_v0=np.zeros((0, 2)), s_n0=np.zeros((0, 2)),
                   s_cons=np.zeros(0, np.uint8), s_dp=dp / 2)


@pytest.mark.parametrize("eta, ratio", [(0.0, 2.5), (0.0, 3.2), (0.05, 1.7)])
def test_automatic_advection_steps_follow_the_criterion(eta, ratio):
    """Reading F3 on a block whose speed stays |U| (checked): with a fixed dt
    an advection step lasts while the steps taken in it sum to at most
    dt_ad = 0.25 min(h / |U|, h^2 / nu), i.e. floor(dt_ad / dt) + 1 steps, so
    the configuration is rebuilt every that many steps; the viscous limit
    takes over when h^2 / nu is the smaller term."""
    U = (0.7, 0.4)
    case = _translating_block(U, eta)
    s = O.OracleSim(case)
    s.set_advection_cadence("auto")
    h = 1.3 * case.f_dp
    speed = float(np.hypot(*U))
    nu = eta / case.f_rho0
    dt_ad = 0.25 * min(h / speed, h * h / nu if nu > 0 else np.inf)
    if eta > 0:
        assert h * h / nu < h / speed   # the viscous term decides here
    dt = dt_ad / ratio
    m = int(np.floor(ratio)) + 1
    for _ in range(4 * m):
        s.step(dt, 1)
    assert np.allclose(s.f_v, np.asarray(U), rtol=0, atol=1e-13)
    assert s.rebuilds == list(range(0, 4 * m, m))


def test_automatic_advection_step_takes_the_smallest_criterion_over_it():
    """An advection step that starts at rest has dt_ad = infinity (no
    viscosity); it ends once the criterion at a later step's maximum is
    exceeded by the time taken since the rebuild."""
    case = _translating_block((0.0, 0.0), 0.0)
    s = O.OracleSim(case)
    s.set_advection_cadence(0)
    dt = 1e-3
    for _ in range(3):
        s.step(dt, 1)
    assert s.rebuilds == [0]        # at rest: held
    s.f_v[:] = (5.0, 0.0)           # now moving: dt_ad = 0.25 h / 5 = 1.625e-3
    for _ in range(3):
        s.step(dt, 1)
    # step 3 starts from the last step's maximum (0: still held, 4 ms taken);
    # step 4 starts from 5: dt_ad drops to 1.625 ms < 5 ms taken, so step 5 rebuilds
    assert s.rebuilds == [0, 5]


# --------------------------------------------------------------------------
# The OpenMP build that times the oracle on many cores gives the same bits
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny_box", "tiny_box_3d", "channel_flag"])
def test_threaded_oracle_build_is_bit_identical(name):
    case = getattr(fc, name)(seed=6)
    a, b = O.OracleSim(case), O.OracleSim(case, threaded=True)
    dt, _, dts = a.suggest_dt()
    K = a.substeps(dt, dts)
    for _ in range(4):
        da, db = a.step(dt, K), b.step(dt, K)
    for k in ("f_r", "f_v", "f_rho", "f_drho", "f_dvdt", "s_r", "s_v", "s_F", "s_fF", "s_vbar", "s_abar", "s_nrm"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    for k in ("mom_fs_fluid", "mom_fs_solid"):
        assert np.array_equal(da[k], db[k]), k
    assert da["abs_fs"] == db["abs_fs"]

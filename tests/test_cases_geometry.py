"""The seeded input generators build the geometries they describe: the
venous valve's two clamped leaflets (Section 4.3) and the flag channel's
Table 1 spacings (Section 4.1)."""
import numpy as np
import pytest
from scipy import spatial

import fsi_cases as fc


@pytest.mark.parametrize("wo", [1.0, 10.0])
def test_venous_valve_leaflets(wo):
    c = fc.venous_valve(seed=0, wo=wo)
    H, L = c.meta["DH"], c.meta["L"]
    b, dpS = 0.2e-3, c.s_dp
    assert dpS == pytest.approx(b / 4) and c.f_dp == pytest.approx(2 * dpS)
    n = c.ns // 2
    assert c.ns == 2 * n and int(c.s_cons.sum()) == 2 * 4 * 4     # 4 rows clamped, 4 through the thickness
    bottom, top = c.s_r0[:n], c.s_r0[n:]
    # mirror images about mid-height
    assert np.allclose(np.sort(bottom[:, 1]), np.sort(H - top[:, 1]), atol=4e-3 * dpS)
    assert np.allclose(np.sort(bottom[:, 0]), np.sort(top[:, 0]), atol=4e-3 * dpS)
    # the observer is on the top leaflet's free end, next to its centre line
    assert c.tip >= n and c.s_r0[c.tip, 1] > H / 2
    root_top = np.array([0.3 * L, H])
    th = np.radians(60.0)
    axis, across = np.array([np.cos(th), -np.sin(th)]), np.array([np.sin(th), np.cos(th)])
    xi, eta = (top - root_top) @ axis, (top - root_top) @ across
    k = c.tip - n
    assert xi[k] > xi.max() - 0.01 * dpS and abs(abs(eta[k]) - 0.5 * dpS) < 0.01 * dpS
    # clamped particles lie inside the walls, free ones inside the channel
    free = c.s_cons == 0
    assert np.all((c.s_r0[~free, 1] < 0.5 * dpS) | (c.s_r0[~free, 1] > H - 0.5 * dpS))
    assert np.all((c.s_r0[free, 1] > -dpS) & (c.s_r0[free, 1] < H + dpS))
    # no fluid particle inside a leaflet; fluid inside the channel
    d, _ = spatial.cKDTree(c.s_r0).query(c.f_r)
    assert d.min() > 0.5 * dpS
    assert c.f_r[:, 0].min() >= 0 and c.f_r[:, 0].max() < L and c.f_r[:, 1].min() > 0 and c.f_r[:, 1].max() < H
    # unit outward normals; the Womersley inflow and the viscosity that gives Wo
    assert np.allclose(np.linalg.norm(c.s_n0, axis=1), 1.0)
    assert c.inflow_profile == 2 and c.inflow_period == 0.6 and c.inflow_wo == wo
    w = 2 * np.pi / c.inflow_period
    assert (H / 2) * np.sqrt(w * c.f_rho0 / c.f_eta) == pytest.approx(wo)


@pytest.mark.parametrize("ratio", [1, 2])
def test_flag_channel_table1_spacings(ratio):
    """Table 1: dp_S is a quarter of the flag's thickness and dp_F = ratio dp_S."""
    D = 0.1
    c = fc.channel_flag(seed=0, dpF=ratio * D * 0.2 / 4, ratio=ratio)
    assert c.s_dp == pytest.approx(0.2 * D / 4)
    assert c.f_dp == pytest.approx(ratio * c.s_dp)
    free = c.s_r0[c.s_cons == 0]
    # the flag is four solid particles thick
    assert len(np.unique(np.floor((free[:, 1] - 2 * D) / c.s_dp))) == 4

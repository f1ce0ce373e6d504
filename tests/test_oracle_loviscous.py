"""Pins of the low-order level's first-order viscous flux (lo_viscous; the
reading of Section 3's "first-order finite volume scheme" for viscous
flow, needed on wall cells thinner than the viscous length, where the
inviscid KFVS correction overshoots the viscous high-order operator).

On an orthogonal mesh the thin-layer normal gradient (u_r - u_l) / delta
is exact for a linear field, so plane Couette flow u = a y (2-D) or
u = a z (3-D) between a wall at rest and a wall moving with the flow,
uniform rho and p, gives in closed form the viscous part of the low-order
residual R_lo(lo_viscous) - R_lo(inviscid): the shear stress mu a is the
same on every face, walls included (the no-slip ghost continues the
linear profile through the wall at twice the centre distance), so every
cell's viscous momentum balance is 0 and its energy gains the shear work
mu a^2 |Omega|.  A wrong sign, a missing Stokes term, a ghost distance off
by two or a wrong face velocity in the work term fails one of them.  The
FAS fixed point stays the high-order one."""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact

GAM = 1.4
P0 = 1.0 / GAM


def viscous_part(s_visc, s_inv, U):
    return s_visc.lo_residual(U) - s_inv.lo_residual(U)


@pytest.mark.parametrize("a", [0.2, -0.35])
def test_couette_viscous_low_order_residual_2d(oracle_lib, a):
    O = oracle_lib
    mu, n = 0.03, 6
    mesh = MG.box(n, n, 0.0, 1.0, 0.0, 1.0, cells="quad", tags=(0, 1, 2, 1))
    om = O.OracleMesh(mesh)
    vol, xc = om.geometry()
    spec = dict(gamma=GAM, mu=mu, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.0, 0.0), p=P0),
                                       dict(kind="noslip", uw=(a, 0.0))])
    U = exact.cons_from_prim(GAM, np.ones(mesh.n_cells), a * xc[:, 1], np.zeros(mesh.n_cells),
                             np.full(mesh.n_cells, P0))
    Rv = viscous_part(O.OracleSolver(om, dict(spec, lo_viscous=1)), O.OracleSolver(om, spec), U)
    h = 1.0 / n
    side = (xc[:, 0] < h) | (xc[:, 0] > 1 - h)       # far-field sides: ghost = the free stream at rest
    walls = (xc[:, 1] < h) | (xc[:, 1] > 1 - h)
    assert (walls & ~side).sum() == 2 * (n - 2)
    mid = ~side                                       # interior and wall cells
    np.testing.assert_allclose(Rv[mid, :3], 0.0, atol=1e-15)
    np.testing.assert_allclose(Rv[mid, 3], mu * a * a * vol[mid], rtol=1e-12)
    assert np.abs(Rv[:, 0]).max() == 0.0         # no viscous mass flux
    # the far-field sides see a jump to the fluid at rest: a real force there
    assert np.abs(Rv[side & ~walls, 1]).min() > 1e-4


def test_couette_viscous_low_order_residual_3d():
    from oracle import oracle3 as O3
    O3.build()
    mu, a, n = 0.02, 0.3, 4
    mesh = MG.box3(n, n, n, cells="hex", tags=(1, 1, 1, 1, 0, 2))
    om = O3.OracleMesh3(mesh)
    vol, xc, _ = om.geometry()
    spec = dict(gamma=GAM, mu=mu, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.0, 0.0, 0.0), p=P0),
                                       dict(kind="noslip", uw=(a, 0.0, 0.0))])
    u = a * xc[:, 2]
    U = np.column_stack([np.ones(mesh.n_cells), u, 0 * u, 0 * u, P0 / (GAM - 1) + 0.5 * u * u])
    Rv = O3.OracleSolver3(om, dict(spec, lo_viscous=1)).lo_residual(U) - O3.OracleSolver3(om, spec).lo_residual(U)
    h = 1.0 / n
    walls = (xc[:, 2] < h) | (xc[:, 2] > 1 - h)
    side = (xc[:, 0] < h) | (xc[:, 0] > 1 - h) | (xc[:, 1] < h) | (xc[:, 1] > 1 - h)
    mid = ~side
    assert (walls & mid).sum() > 0 and (~walls & mid).sum() > 0
    np.testing.assert_allclose(Rv[mid, :4], 0.0, atol=1e-15)
    np.testing.assert_allclose(Rv[mid, 4], mu * a * a * vol[mid], rtol=1e-12)


def test_fas_fixed_point_with_viscous_low_order(oracle_lib):
    """The viscous low-order flux changes the correction, not the fixed
    point: a V-cycle-converged state is left unchanged by the explicit
    high-order step (viscous cylinder, Re 38)."""
    O = oracle_lib
    mesh = MG.cylinder(24, 4, 6, growth=1.2, R_far=5.0)
    ma = 0.38
    spec = dict(gamma=GAM, mu=0.01, cfl_hi=0.4, lo_viscous=1,
                bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    s = O.OracleSolver(O.OracleMesh(mesh), spec)
    W0 = np.tile(exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1 / GAM), (mesh.n_cells, 1))
    s.set_state(W0)
    res = s.pmg_cycles(500)
    assert res[-1] < 1e-14, res[-5:]
    W, _ = s.get_state()
    s.highorder_step()
    W2, _ = s.get_state()
    assert np.abs(W2 - W).max() < 1e-12


def _box2(O, mu, n=6):
    mesh = MG.box(n, n, 0.0, 1.0, 0.0, 1.0, cells="quad", tags=(0, 0, 0, 0))
    om = O.OracleMesh(mesh)
    vol, xc = om.geometry()
    spec = dict(gamma=GAM, mu=mu, bcs=[dict(kind="farfield", rho=1.0, u=(0.0, 0.0), p=P0)])
    h = 1.0 / n
    inner = (xc[:, 0] > h) & (xc[:, 0] < 1 - h) & (xc[:, 1] > h) & (xc[:, 1] < 1 - h)
    return om, vol, xc, spec, inner


def test_stokes_term_and_heat_flux_2d(oracle_lib):
    """Normal strain u = (0, b y): the normal stress is (4/3) mu b on every
    face (Stokes' hypothesis), so interior cells gain the work
    (4/3) mu b^2 |Omega| and no momentum.  A quadratic temperature
    T = T0 + c y^2 at rest: the face difference of T is exact at the face
    midpoints, so interior cells gain kappa T'' |Omega| = kappa 2c |Omega|
    (kappa = mu gamma / (gamma - 1), Pr = 1) and no momentum."""
    O = oracle_lib
    mu, b, c = 0.02, 0.3, 0.4
    om, vol, xc, spec, inner = _box2(O, mu)
    sv, si = O.OracleSolver(om, dict(spec, lo_viscous=1)), O.OracleSolver(om, spec)
    n = vol.size
    U = exact.cons_from_prim(GAM, np.ones(n), np.zeros(n), b * xc[:, 1], np.full(n, P0))
    Rv = viscous_part(sv, si, U)
    np.testing.assert_allclose(Rv[inner, :3], 0.0, atol=1e-15)
    np.testing.assert_allclose(Rv[inner, 3], 4.0 / 3.0 * mu * b * b * vol[inner], rtol=1e-12)
    T = P0 + c * xc[:, 1] ** 2
    U = exact.cons_from_prim(GAM, np.ones(n), np.zeros(n), np.zeros(n), T)     # rho = 1: p = T
    Rv = viscous_part(sv, si, U)
    kappa = mu * GAM / (GAM - 1.0)
    np.testing.assert_allclose(Rv[inner, :3], 0.0, atol=1e-15)
    np.testing.assert_allclose(Rv[inner, 3], kappa * 2.0 * c * vol[inner], rtol=1e-12)

"""Pins of the oracle's wall loads (the surface quantities behind Section
4's Cd, Cl, Cp and Cf): the momentum part of the high-order face flux F0
through the faces of one boundary tag, per unit length (2-D) or area (3-D).

Closed forms that fix it:
* fluid at rest at uniform pressure p: the traction is p n on every wall
  face (slip and no-slip), and sum S n vanishes over a closed boundary;
* plane Couette flow u = a y (2-D) or u = a z (3-D) between a wall at rest
  and a wall moving with u = a, uniform rho and p: with Pr = 1 the
  gas-kinetic flux reproduces the Navier-Stokes stress, so the traction on
  the wall at rest is (mu a, -p) and on the moving wall (-mu a, p), in 3-D
  (mu a, 0, -p) and (-mu a, 0, p).  A wrong sign of the viscous term, a
  normal into the fluid or a dropped Gauss point fails one of these.
"""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact
from tests.test_oracle3 import tet_quad

GAM = 1.4
P0 = 1.0 / GAM


def mesh2():
    return MG.box(8, 8, 0.0, 1.0, 0.0, 1.0, jitter=0.2, seed=4, cells="mixed",
                  quad_mask=lambda i, j: (i + j) % 3 == 0, tags=(0, 1, 2, 1))


def test_rest_state_traction_is_pressure_2d(oracle_lib):
    O = oracle_lib
    mesh = mesh2()
    spec = dict(gamma=GAM, mu=0.02, bcs=[dict(kind="noslip"), dict(kind="slip"), dict(kind="slip")])
    W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, P0), (mesh.n_cells, 1))
    s = O.OracleSolver(O.OracleMesh(mesh), spec)
    s.set_state(W)
    total = np.zeros(2)
    for tag in (0, 1, 2):
        d = s.wall_loads(tag)
        assert len(d["S"]) > 0
        np.testing.assert_allclose(d["traction"], P0 * d["n"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(np.linalg.norm(d["n"], axis=1), 1.0, atol=1e-14)
        total += (d["S"][:, None] * d["n"]).sum(0)
    assert np.abs(total).max() < 1e-14


@pytest.mark.parametrize("a", [0.3, -0.2])
def test_couette_traction_2d(oracle_lib, a):
    O = oracle_lib
    mu = 0.05
    mesh = mesh2()
    spec = dict(gamma=GAM, mu=mu, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.0, 0.0), p=P0),
                                       dict(kind="noslip", uw=(a, 0.0))])
    W, Wx = exact.cell_averages(mesh, lambda x, y: exact.cons_from_prim(GAM, 1.0 + 0 * x, a * y, 0 * x,
                                                                        P0 + 0 * x))
    s = O.OracleSolver(O.OracleMesh(mesh), spec)
    s.set_state(W, Wx)
    bottom, top = s.wall_loads(0), s.wall_loads(2)
    assert len(bottom["S"]) == 8 and len(top["S"]) == 8
    np.testing.assert_allclose(bottom["n"], np.tile([0.0, -1.0], (8, 1)), atol=1e-15)
    np.testing.assert_allclose(bottom["traction"], np.tile([mu * a, -P0], (8, 1)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(top["traction"], np.tile([-mu * a, P0], (8, 1)), rtol=0, atol=1e-13)
    # face centres on the walls, lengths summing to the wall length
    np.testing.assert_allclose(bottom["x"][:, 1], 0.0, atol=1e-15)
    assert abs(bottom["S"].sum() - 1.0) < 1e-14 and abs(top["S"].sum() - 1.0) < 1e-14


@pytest.fixture(scope="module")
def O3():
    from oracle import oracle3
    oracle3.build()
    return oracle3


def test_couette_traction_3d(O3):
    mu, a = 0.04, 0.25
    mesh = MG.box3(3, 3, 4, jitter=0.15, seed=5, cells="tet", tags=(1, 1, 1, 1, 0, 2))

    def field(x):
        u = a * x[2]
        return np.array([1.0, u, 0.0, 0.0, P0 / (GAM - 1) + 0.5 * u * u])
    W = np.zeros((mesh.n_cells, 5))
    Wx = np.zeros((mesh.n_cells, 3, 5))
    for c in range(mesh.n_cells):
        P = mesh.nodes[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]]
        W[c] = [tet_quad(P, lambda x, v=v: field(x)[v]) for v in range(5)]
        zc = tet_quad(P, lambda x: x[2])
        Wx[c, 2] = [0.0, a, 0.0, 0.0, a * a * zc]       # mean gradient of the linear / quadratic parts
    spec = dict(gamma=GAM, mu=mu, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.0, 0.0, 0.0), p=P0),
                                       dict(kind="noslip", uw=(a, 0.0, 0.0))])
    s = O3.OracleSolver3(O3.OracleMesh3(mesh), spec)
    s.set_state(W, Wx)
    bottom, top = s.wall_loads(0), s.wall_loads(2)
    nb, nt = len(bottom["S"]), len(top["S"])
    assert nb == nt == 2 * 3 * 3
    np.testing.assert_allclose(bottom["traction"], np.tile([mu * a, 0.0, -P0], (nb, 1)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(top["traction"], np.tile([-mu * a, 0.0, P0], (nt, 1)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(bottom["x"][:, 2], 0.0, atol=1e-15)
    assert abs(bottom["S"].sum() - 1.0) < 1e-13

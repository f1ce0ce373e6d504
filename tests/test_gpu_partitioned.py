"""The partitioned sweep (CGKS_SWEEP_PARTITIONED) against the oracle's
'partitioned_colour' order: the reverse Cuthill-McKee order cut into
ceil(n / sweep_part_cells) partitions, colour classes inside each, the
exchange between partitions lagged by one sweep (the paper's threaded
sweep of Section 3 made deterministic).  One thread-block cluster per
partition on the GPU.  FP64 within 1e-12 relative L2 per V-cycle, mixed
within 1e-5; residual histories within 1e-9 (FP64)."""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact
from tests.test_gpu_parity import TOL, case, libs, rel  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu
GAM = 1.4


def pair_part(libs, mesh, spec, state, part_cells, precision="fp64"):
    cgks, O = libs
    n_parts = math.ceil(mesh.n_cells / part_cells)
    g = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision=precision, sweep_order="partitioned",
                                          sweep_part_cells=part_cells))
    o = O.OracleSolver(O.OracleMesh(mesh), dict(spec, sweep_order="partitioned_colour", n_parts=n_parts))
    g.set_state(*state)
    o.set_state(*state)
    return g, o, n_parts


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,part_cells", [("cavity8", 64), ("mixed_slip_farfield", 64),
                                             ("cylinder_viscous", 64), ("linear_fallback", 64)])
def test_partitioned_cycles_match_oracle(libs, name, part_cells, precision):
    mesh, spec, state = case(name)
    g, o, n_parts = pair_part(libs, mesh, spec, state, part_cells, precision)
    assert n_parts >= 2
    hg, ho = g.pmg_cycle(4), o.pmg_cycles(4)
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    tol = TOL if precision == "fp64" else 1e-5
    assert rel(Wg, Wo) < tol, rel(Wg, Wo)
    if precision == "fp64":
        assert rel(Xg, Xo) < TOL, rel(Xg, Xo)
        np.testing.assert_allclose(hg, ho, rtol=1e-9)
    # two launches per implicit step (n_sweeps = 2), no colour launches
    assert g.launches_per_call(True) < cgks_colour_launches(libs, mesh, spec)


def cgks_colour_launches(libs, mesh, spec):
    cgks, _ = libs
    s = cgks.Solver(cgks.Mesh(mesh), spec)
    return s.launches_per_call(True)


def test_partitioned_differs_from_colour_order(libs):
    """The lag is real: with several partitions the V-cycle differs from the
    colour-class order (and from the oracle's colour order), while one
    partition reproduces the colour-class order to rounding."""
    cgks, O = libs
    mesh, spec, state = case("cylinder_viscous")
    g1, _, _ = pair_part(libs, mesh, spec, state, 100000)
    c = cgks.Solver(cgks.Mesh(mesh), spec)
    c.set_state(*state)
    h1, hc = g1.pmg_cycle(3), c.pmg_cycle(3)
    assert rel(g1.get_state()[0], c.get_state()[0]) < TOL
    gp, _, _ = pair_part(libs, mesh, spec, state, 64)
    gp.pmg_cycle(3)
    assert rel(gp.get_state()[0], c.get_state()[0]) > 1e-9


def test_cavity_2048_partitioned_eight_parts(libs):
    """The 2048-cell cavity of the first configuration, 256-cell partitions:
    eight clusters, five V-cycles."""
    mesh = MG.cavity(32)
    spec = dict(gamma=GAM, mu=0.15 / 1000, cfl_hi=0.5,
                bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(0.15, 0.0))])
    W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
    g, o, n_parts = pair_part(libs, mesh, spec, (W, None), 256)
    assert n_parts == 8
    hg, ho = g.pmg_cycle(5), o.pmg_cycles(5)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    assert rel(g.get_state()[0], o.get_state()[0]) < TOL


def test_cylinder_57344_partitioned_default_parts(libs):
    """The benchmark's 57,344-cell cylinder with the default 2048-cell
    partitions (28 clusters of 8 CTAs), two V-cycles from a perturbed
    state."""
    from tests.test_gpu_developed import perturbed
    mesh = MG.cylinder(256, 32, 96)
    ma = 0.38
    spec = dict(gamma=GAM, mu=0.0, cfl_hi=0.4,
                bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    W, Wx = perturbed(mesh, (ma, 0.0), 0.04, seed=58)
    g, o, n_parts = pair_part(libs, mesh, spec, (W, Wx), 2048)
    assert n_parts == 28
    hg, ho = g.pmg_cycle(2), o.pmg_cycles(2)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    assert rel(g.get_state()[0], o.get_state()[0]) < TOL


def test_partitioned_rejections(libs):
    cgks, _ = libs
    mesh, spec, state = case("cavity8")
    for bad in (dict(sweep_part_cells=32), dict(low_order_fused=1)):
        with pytest.raises(cgks.CgksError):
            cgks.Solver(cgks.Mesh(mesh), dict(spec, sweep_order="partitioned", **bad))
    m3 = MG.box3(2, 2, 2, cells="tet", tags=(0, 0, 0, 0, 0, 0))
    with pytest.raises(cgks.CgksError):
        cgks.Solver(cgks.Mesh(m3), dict(gamma=GAM, sweep_order="partitioned",
                                        bcs=[dict(kind="farfield", rho=1.0, u=(0.1, 0.0, 0.0), p=1 / GAM)]))

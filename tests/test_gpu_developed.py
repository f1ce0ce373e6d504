"""Parity on developed flow at full size (FP64 against the CPU oracle).

The 57,344-cell cylinder of the benchmark, started from the free stream
plus a seeded smooth perturbation (so every cell carries gradients from the
first cycle), run for 20 V-cycles in the launch configuration the benchmark
times; and a 3-D sphere shell of 30,720 cells (icosphere level 3, 12 prism
and 4 split-tet layers) for 5 V-cycles.  Residual histories within 1e-9,
the fields within 1e-12 relative L2 (W) per the FP64 bar."""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact

pytestmark = pytest.mark.gpu
GAM = 1.4
TOL = 1e-12


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def node_centroids(mesh):
    ptr = mesh.cell_ptr
    return np.add.reduceat(mesh.nodes[mesh.cell_nodes], ptr[:-1], axis=0) / np.diff(ptr)[:, None]


def perturbed(mesh, vel, amp, seed):
    """Free stream plus a smooth seeded perturbation at the cell centres,
    its analytic gradient as the cell gradients."""
    rng = np.random.default_rng(seed)
    dim = mesh.nodes.shape[1]
    k = rng.uniform(0.8, 2.0, dim)
    ph = rng.uniform(0.0, 1.0, dim)
    x = node_centroids(mesh)

    def f(x):
        s = amp * np.prod([np.sin(k[d] * x[:, d] + ph[d]) for d in range(dim)], axis=0)
        rho, p = 1.0 + s, (1.0 + 0.7 * s) / GAM
        u = [vel[d] + (0.5, -0.3, 0.2)[d] * s for d in range(dim)]
        ke = 0.5 * rho * sum(ud * ud for ud in u)
        return np.stack([rho] + [rho * ud for ud in u] + [p / (GAM - 1) + ke], -1)
    h = 1e-6
    Wx = np.stack([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(dim)], axis=1)
    return f(x), Wx


@pytest.fixture(scope="module")
def libs(oracle_lib):
    from oracle import oracle3
    from paper_2109_09965_gb300 import cgks
    oracle3.build()
    cgks.lib()
    return cgks, oracle_lib, oracle3


def test_cylinder_57344_developed_flow_20_cycles(libs):
    cgks, O, _ = libs
    mesh = MG.cylinder(256, 32, 96)
    assert mesh.n_cells == 57344
    ma = 0.38
    spec = dict(gamma=GAM, mu=0.0, cfl_hi=0.4, cfl_lo=1000.0, n_implicit=6, n_sweeps=2, time_scheme="S1O2",
                bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    W, Wx = perturbed(mesh, (ma, 0.0), 0.04, seed=57)
    g = cgks.Solver(cgks.Mesh(mesh), spec)
    o = O.OracleSolver(O.OracleMesh(mesh), spec)
    g.set_state(W, Wx)
    o.set_state(W, Wx)
    hg, ho = g.pmg_cycle(20), o.pmg_cycles(20)
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    eW, eX = rel(Wg, Wo), rel(Xg, Xo)
    print(f"57k developed: rel W {eW:.2e}  Wx {eX:.2e}  Res {np.abs(hg / ho - 1).max():.2e}")
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    assert eW < TOL, eW
    assert eX < TOL, eX
    assert rel(W, Wo) > 1e-4          # the field did change


def test_sphere_shell_30720_developed_flow_5_cycles(libs):
    cgks, _, O3 = libs
    mesh = MG.sphere(3, 12, 4, h0=5e-3, growth=1.35, R_far=5.0)
    assert mesh.n_cells == 30720
    vel = (0.2, 0.0, 0.0)
    spec = dict(gamma=GAM, mu=0.2 / 118, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
    W, Wx = perturbed(mesh, vel, 0.03, seed=30)
    g = cgks.Solver(cgks.Mesh(mesh), spec)
    o = O3.OracleSolver3(O3.OracleMesh3(mesh), spec)
    g.set_state(W, Wx)
    o.set_state(W, Wx)
    hg, ho = g.pmg_cycle(5), o.pmg_cycles(5)
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    eW, eX = rel(Wg, Wo), rel(Xg, Xo)
    print(f"sphere 30720 developed: rel W {eW:.2e}  Wx {eX:.2e}  Res {np.abs(hg / ho - 1).max():.2e}")
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    assert eW < TOL, eW
    assert eX < TOL, eX

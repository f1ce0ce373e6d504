"""3-D GPU path (libcgks, FP64 and mixed) against the 3-D CPU oracle.

Per-iteration relative L2 of W, Wx and R_p0 after explicit steps (S1O2,
S2O4) and V-cycles, on tet / prism / pyramid / hex boxes with far-field,
slip and moving no-slip boundaries and on a small sphere shell.  FP64 bar
1e-12 (same formulas in double; summation order, transcendental rounding
and Gram-Schmidt vs Householder operators differ at O(1e-15) per step);
mixed bar 1e-5 relative over a few steps.
"""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG

pytestmark = pytest.mark.gpu
GAM = 1.4
TOL = 1e-12


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cons3(rho, u, v, w, p):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (GAM - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


def centroids(mesh):
    return np.array([mesh.nodes[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]].mean(0)
                     for c in range(mesh.n_cells)])


def smooth_state(mesh, vel, amp=0.03, seed=0):
    """Free stream plus a smooth seeded perturbation; gradients analytic."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.0, 2.5, 3)
    x = centroids(mesh)

    def f(x):
        s = amp * np.sin(k[0] * x[:, 0] + 0.3) * np.cos(k[1] * x[:, 1]) * np.cos(k[2] * x[:, 2] + 0.1)
        return cons3(1 + s, vel[0] + 0.5 * s, vel[1] - 0.3 * s, vel[2] + 0.2 * s, (1 + 0.7 * s) / GAM)
    W = f(x)
    h = 1e-6
    Wx = np.stack([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
    return W, Wx


def case(name):
    if name == "tet_farfield":
        mesh = MG.box3(3, 3, 2, jitter=0.2, seed=1, cells="tet", tags=(0, 0, 0, 0, 0, 0))
        vel = (0.3, 0.1, -0.1)
        spec = dict(gamma=GAM, mu=0.005, bcs=[dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, vel)
    if name == "prism_walls":
        mesh = MG.box3(3, 2, 3, jitter=0.2, seed=2, cells="prism", tags=(2, 2, 2, 2, 0, 1))
        vel = (0.2, 0.0, 0.0)
        spec = dict(gamma=GAM, mu=0.01,
                    bcs=[dict(kind="slip"), dict(kind="noslip", uw=(0.1, 0.05, 0.0)),
                         dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, vel, seed=3)
    if name == "pyramid_noslip":
        mesh = MG.box3(2, 2, 2, jitter=0.1, seed=4, cells="pyramid", tags=(1, 1, 1, 1, 0, 1))
        vel = (0.1, 0.2, 0.0)
        spec = dict(gamma=GAM, mu=0.02,
                    bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, vel, seed=5)
    if name == "hex_slip":
        mesh = MG.box3(3, 3, 3, jitter=0.15, seed=6, cells="hex", tags=(1, 1, 0, 0, 1, 1))
        vel = (0.25, 0.0, 0.1)
        spec = dict(gamma=GAM, mu=0.0, bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, vel, seed=7)
    if name == "sphere":
        mesh = MG.sphere(1, 4, 2, h0=0.02, growth=1.4, R_far=4.0)
        vel = (0.2, 0.0, 0.0)
        spec = dict(gamma=GAM, mu=0.2 / 118,
                    bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
        W = np.tile(cons3(1.0, *vel, 1 / GAM), (mesh.n_cells, 1))
        return mesh, spec, (W, np.zeros((mesh.n_cells, 3, 5)))
    raise KeyError(name)


CASES = ["tet_farfield", "prism_walls", "pyramid_noslip", "hex_slip", "sphere"]


@pytest.fixture(scope="module")
def libs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from oracle import oracle3 as O3
    from paper_2109_09965_gb300 import cgks
    O3.build()
    cgks.lib()
    return cgks, O3


def pair(libs, name, **over):
    cgks, O3 = libs
    mesh, spec, (W, Wx) = case(name)
    spec = dict(spec, **over)
    s = cgks.Solver(cgks.Mesh(mesh), spec)
    s.set_state(W, Wx)
    o = O3.OracleSolver3(O3.OracleMesh3(mesh), spec)
    o.set_state(W, Wx)
    return s, o


@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("name", CASES)
def test_explicit_steps_match_oracle(libs, name, scheme):
    s, o = pair(libs, name, time_scheme=scheme)
    for k in range(3):
        dg = s.highorder_step()
        do = o.highorder_step()
        assert abs(dg - do) <= 1e-13 * do
        Wg, Xg = s.get_state()
        Wo, Xo = o.get_state()
        assert rel(Wg, Wo) < TOL, (k, rel(Wg, Wo))
        assert rel(Xg, Xo) < TOL, (k, rel(Xg, Xo))
        rg, _ = s.residual()
        assert abs(rg - o.residual()) <= 1e-9 * o.residual()


@pytest.mark.parametrize("name", CASES)
def test_pmg_cycles_match_oracle(libs, name):
    s, o = pair(libs, name)
    hg = s.pmg_cycle(3)
    ho = o.pmg_cycles(3)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    Wg, Xg = s.get_state()
    Wo, Xo = o.get_state()
    assert rel(Wg, Wo) < TOL, rel(Wg, Wo)
    assert rel(Xg, Xo) < TOL, rel(Xg, Xo)
    assert rel(s.rp0(), o.get_rp0()) < 1e-10


def test_graph_replay_is_bitwise_equal_to_launches(libs):
    cgks, _ = libs
    mesh, spec, (W, Wx) = case("prism_walls")
    out = []
    for g in (1, 0):
        s = cgks.Solver(cgks.Mesh(mesh), dict(spec, use_graph=g, autotune=0))
        s.set_state(W, Wx)
        s.pmg_cycle(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("name", ["tet_farfield", "prism_walls", "sphere"])
def test_mixed_precision_tracks_fp64(libs, name):
    cgks, O3 = libs
    mesh, spec, (W, Wx) = case(name)
    o = O3.OracleSolver3(O3.OracleMesh3(mesh), spec)
    o.set_state(W, Wx)
    o.explicit_steps(2)
    o.pmg_cycles(2)
    s = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision="mixed"))
    s.set_state(W, Wx)
    s.explicit_steps(2)
    s.pmg_cycle(2)
    Wg, _ = s.get_state()
    Wo, _ = o.get_state()
    assert rel(Wg, Wo) < 1e-5, rel(Wg, Wo)


def test_sphere_config_mesh_runs(libs):
    """The configured sphere construction at level 2 (realistic prism
    stack): V-cycles run without diverging and reduce Res."""
    cgks, _ = libs
    mesh = MG.sphere(2, 12, 4, h0=5e-3, growth=1.35, R_far=5.0)
    vel = (0.2, 0.0, 0.0)
    spec = dict(gamma=GAM, mu=0.2 / 118, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
    for prec in ("fp64", "mixed"):
        s = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision=prec))
        s.set_state(np.tile(cons3(1.0, *vel, 1 / GAM), (mesh.n_cells, 1)))
        h = s.pmg_cycle(60)
        assert np.all(np.isfinite(h)) and h[-1] < 0.1 * h[0], (prec, h[::10])


@pytest.mark.parametrize("name", ["prism_walls", "sphere"])
def test_lf_low_level_matches_oracle(libs, name):
    s, o = pair(libs, name, flux_lo="lf")
    hg = s.pmg_cycle(3)
    ho = o.pmg_cycles(3)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    Wg, Xg = s.get_state()
    Wo, Xo = o.get_state()
    assert rel(Wg, Wo) < TOL, rel(Wg, Wo)
    assert rel(Xg, Xo) < TOL, rel(Xg, Xo)

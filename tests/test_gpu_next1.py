"""Full gas-kinetic flux (Eq. (2nd-flux)), compact WENO weights and the
Dirichlet / supersonic-outflow boundaries on the GPU against the oracle,
through the C ABI.

The shock reflection problem of Section 4 (reflective bottom wall,
supersonic outflow on the right, Dirichlet states on the left and top,
inviscid, full flux, WENO with epsilon 1e-2 and 1e-6) on a coarse copy of
its grid and at the paper's 120 x 30; a viscous smooth case with the full
flux; the free-stream check through the new boundaries.  FP64 bar 1e-12
relative L2 per step (the same formulas in double precision on both sides;
the WENO smoothness indicators are taken by a quadrature in the oracle and
by cell moments on the GPU, equal to rounding); the mixed path (FP32
reconstruction and fluxes) within 1e-4 over a few steps.
"""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests.test_gpu_parity import case, check, pair, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs(oracle_lib):
    import torch
    from paper_2109_09965_gb300 import cgks
    assert torch.cuda.is_available()
    cgks.lib()
    return cgks, oracle_lib


def shock_case(nx, ny, eps, weno_vars="conservative"):
    mesh, spec, W0 = MG.shock_reflection_case(nx, ny, weno_eps=eps, weno_vars=weno_vars)
    return mesh, spec, (W0, np.zeros((mesh.n_cells, 2, 4)))


def advance_oracle(O, mesh, spec, state, n):
    """A developed (non-uniform) starting state: n oracle V-cycles."""
    o = O.OracleSolver(O.OracleMesh(mesh), spec)
    o.set_state(*state)
    o.pmg_cycles(n)
    return o.get_state()


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("eps", [1e-2, 1e-6])
def test_shock_reflection_explicit_steps_match_oracle(libs, eps, scheme, weno_vars):
    cgks, O = libs
    mesh, spec, state = shock_case(24, 6, eps, weno_vars)
    spec = dict(spec, time_scheme=scheme)
    state = advance_oracle(O, mesh, spec, state, 20)
    g, o = pair(libs, mesh, spec, state)
    for k in range(4):
        rg = g.explicit_steps(1)
        ro = o.explicit_steps(1)
        check(g, o, f"step {k + 1}")
        assert abs(rg[0] - ro[0]) <= 1e-9 * abs(ro[0])


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("eps", [1e-2, 1e-6])
def test_shock_reflection_cycles_match_oracle(libs, eps, scheme, weno_vars):
    cgks, O = libs
    mesh, spec, state = shock_case(24, 6, eps, weno_vars)
    spec = dict(spec, time_scheme=scheme)
    g, o = pair(libs, mesh, spec, state)
    for k in range(4):
        rg = g.pmg_cycle(1)
        ro = o.pmg_cycles(1)
        check(g, o, f"cycle {k + 1}")
        assert abs(rg[0] - ro[0]) <= 1e-9 * abs(ro[0]), (rg, ro)


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
@pytest.mark.parametrize("flux_lo", ["kfvs", "lf"])
@pytest.mark.parametrize("name", ["cavity8", "mixed_slip_farfield"])
def test_viscous_full_flux_with_weno_matches_oracle(libs, name, flux_lo, weno_vars):
    mesh, spec, state = case(name)
    spec = dict(spec, flux_hi="full", weno_eps=1e-6, tau_c1=0.05, tau_c2=2.0, flux_lo=flux_lo, weno_vars=weno_vars)
    g, o = pair(libs, mesh, spec, state)
    for k in range(2):
        g.explicit_steps(1)
        o.explicit_steps(1)
        check(g, o, f"step {k + 1}")
    hg, ho = g.pmg_cycle(2), o.pmg_cycles(2)
    check(g, o, "cycles")
    np.testing.assert_allclose(hg, ho, rtol=1e-9)


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
def test_shock_reflection_full_grid_matches_oracle(libs, weno_vars):
    """The paper's 120 x 30 grid: two V-cycles from the uniform start."""
    mesh, spec, state = shock_case(120, 30, 1e-2, weno_vars)
    g, o = pair(libs, mesh, spec, state)
    hg, ho = g.pmg_cycle(2), o.pmg_cycles(2)
    check(g, o, "120x30")
    np.testing.assert_allclose(hg, ho, rtol=1e-9)


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
def test_shock_reflection_mixed_precision(libs, scheme, weno_vars):
    cgks, O = libs
    mesh, spec, state = shock_case(24, 6, 1e-2, weno_vars)
    spec = dict(spec, time_scheme=scheme)
    state = advance_oracle(O, mesh, spec, state, 20)
    g, o = pair(libs, mesh, dict(spec, precision="mixed"), state)
    g.explicit_steps(2)
    o.explicit_steps(2)
    g.pmg_cycle(2)
    o.pmg_cycles(2)
    Wg, _ = g.get_state()
    Wo, _ = o.get_state()
    assert rel(Wg, Wo) < 1e-4, rel(Wg, Wo)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_supersonic_stream_kept_through_new_boundaries(libs, precision):
    cgks, O = libs
    mesh, spec, W0 = MG.shock_reflection_case(12, 4, weno_eps=1e-6, weno_vars="conservative")
    spec["bcs"][MG.SR_TOP] = dict(spec["bcs"][MG.SR_INFLOW])
    s = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision=precision))
    s.set_state(W0)
    s.explicit_steps(3)
    s.pmg_cycle(2)
    W, Wx = s.get_state()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.abs(W - W0).max() < tol * np.abs(W0).max()


@pytest.mark.parametrize("weno_vars", ["conservative", "characteristic"])
def test_graph_and_plain_launches_agree_bitwise(libs, weno_vars):
    cgks, O = libs
    mesh, spec, state = shock_case(24, 6, 1e-2, weno_vars)
    out = []
    for graph in (0, 1):
        s = cgks.Solver(cgks.Mesh(mesh), dict(spec, use_graph=graph, autotune=0))
        s.set_state(*state)
        h = s.pmg_cycle(5)
        out.append((h, *s.get_state()))
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)

"""GPU (libcgks, FP64) against the CPU oracle, through the C ABI.

Per-iteration relative L2 of W and Wx and of the density residual, bar
1e-12 for the FP64 path: both sides evaluate the same formulas in double
precision and differ only by summation order, libm vs CUDA transcendental
rounding and QR vs Gram-Schmidt operators, all O(1e-15) per step.
"""
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


def smooth_state(mesh, ma, aoa=0.0, amp=0.05, seed=0):
    """Free stream plus a smooth seeded perturbation, with exact gradients."""
    rng = np.random.default_rng(seed)
    kx, ky, ph = rng.uniform(0.5, 2.0, 3)
    x0, x1 = mesh.nodes[:, 0].min(), mesh.nodes[:, 0].max()
    y0, y1 = mesh.nodes[:, 1].min(), mesh.nodes[:, 1].max()
    L = max(x1 - x0, y1 - y0)

    def f(x, y):
        s = amp * np.sin(2 * np.pi * (kx * x + ph) / L) * np.cos(2 * np.pi * ky * y / L)
        rho = 1.0 + s
        u = ma * math.cos(aoa) + 0.5 * s
        v = ma * math.sin(aoa) - 0.3 * s
        return exact.cons_from_prim(GAM, rho, u, v, (1.0 + 0.7 * s) / GAM)
    return exact.cell_averages(mesh, f)


def case(name):
    if name == "cavity8":
        mesh = MG.cavity(8)
        spec = dict(gamma=GAM, mu=0.15 / 100, cfl_hi=0.5,
                    bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(0.15, 0.0))])
        return mesh, spec, smooth_state(mesh, 0.0, amp=0.02)
    if name == "mixed_slip_farfield":
        mesh = MG.box(9, 7, 0.0, 1.5, 0.0, 1.0, jitter=0.2, seed=5, cells="mixed",
                      quad_mask=lambda i, j: (2 * i + j) % 5 == 0, tags=(0, 1, 1, 1))
        spec = dict(gamma=GAM, mu=0.01, cfl_hi=0.4,
                    bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(0.3, 0.0), p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, 0.3)
    if name == "cylinder_inviscid":
        mesh = MG.cylinder(32, 4, 8)
        spec = dict(gamma=GAM, mu=0.0, cfl_hi=0.4,
                    bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(0.38, 0.0), p=1 / GAM)])
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.38, 0.0, 1 / GAM), (mesh.n_cells, 1))
        return mesh, spec, (W, np.zeros((mesh.n_cells, 2, 4)))
    if name == "cylinder_viscous":
        mesh = MG.cylinder(24, 4, 6, growth=1.2, R_far=5.0)
        spec = dict(gamma=GAM, mu=0.01, cfl_hi=0.4,
                    bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.38, 0.0), p=1 / GAM)])
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.38, 0.0, 1 / GAM), (mesh.n_cells, 1))
        return mesh, spec, (W, np.zeros((mesh.n_cells, 2, 4)))
    if name == "linear_fallback":
        # '/' split with far field everywhere: two corner triangles have a
        # single face neighbour and fall back to the linear reconstruction
        mesh = MG.box(6, 6, jitter=0.15, seed=7, cells="slash", tags=(0, 0, 0, 0))
        spec = dict(gamma=GAM, mu=0.005, cfl_hi=0.4,
                    bcs=[dict(kind="farfield", rho=1.0, u=(0.2, 0.1), p=1 / GAM)])
        return mesh, spec, smooth_state(mesh, 0.2, aoa=0.4)
    raise KeyError(name)


CASES = ["cavity8", "mixed_slip_farfield", "cylinder_inviscid", "cylinder_viscous", "linear_fallback"]


@pytest.fixture(scope="module")
def libs(oracle_lib):
    import torch
    from paper_2109_09965_gb300 import cgks
    assert torch.cuda.is_available()
    cgks.lib()
    return cgks, oracle_lib


def pair(libs, mesh, spec, state):
    cgks, O = libs
    g = cgks.Solver(cgks.Mesh(mesh), spec)
    o = O.OracleSolver(O.OracleMesh(mesh), spec)
    g.set_state(*state)
    o.set_state(*state)
    return g, o


def check(g, o, what):
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    e1, e2 = rel(Wg, Wo), rel(Xg, Xo)
    assert e1 < TOL and e2 < TOL, f"{what}: W {e1:.2e} Wx {e2:.2e}"


@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("name", CASES)
def test_explicit_steps_match_oracle(libs, name, scheme):
    mesh, spec, state = case(name)
    spec = dict(spec, time_scheme=scheme)
    g, o = pair(libs, mesh, spec, state)
    dt_g = g.highorder_step()
    dt_o = o.highorder_step()
    assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    check(g, o, "step 1")
    for k in range(4):
        rg = g.explicit_steps(1)
        ro = o.explicit_steps(1)
        check(g, o, f"step {k + 2}")
        assert abs(rg[0] - ro[0]) <= 1e-10 * abs(ro[0]) + 1e-300


@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("name", CASES)
def test_pmg_cycles_match_oracle(libs, name, scheme):
    mesh, spec, state = case(name)
    spec = dict(spec, time_scheme=scheme)
    g, o = pair(libs, mesh, spec, state)
    for k in range(3):
        rg = g.pmg_cycle(1)
        ro = o.pmg_cycles(1)
        check(g, o, f"cycle {k + 1}")
        assert abs(rg[0] - ro[0]) <= 1e-10 * abs(ro[0]), (rg, ro)
        np.testing.assert_allclose(g.rp0(), o.get_rp0(), rtol=0,
                                   atol=TOL * np.abs(o.get_rp0()).max())


def test_loworder_smooth_alone(libs):
    mesh, spec, state = case("mixed_slip_farfield")
    g, o = pair(libs, mesh, spec, state)
    g.highorder_step()
    o.highorder_step()
    g.loworder_smooth()
    o.loworder_smooth()
    check(g, o, "smoother")


def test_many_cycles_and_history(libs):
    """20 cycles in one call (CUDA graph) against the oracle, residual history
    element by element."""
    mesh, spec, state = case("cylinder_viscous")
    g, o = pair(libs, mesh, spec, state)
    rg = g.pmg_cycle(20)
    ro = o.pmg_cycles(20)
    check(g, o, "20 cycles")
    np.testing.assert_allclose(rg, ro, rtol=1e-9)


def test_graph_and_plain_launches_agree_bitwise(libs):
    cgks, _ = libs
    mesh, spec, state = case("cavity8")
    a = cgks.Solver(cgks.Mesh(mesh), dict(spec, use_graph=1, autotune=0))
    b = cgks.Solver(cgks.Mesh(mesh), dict(spec, use_graph=0, autotune=0))
    a.set_state(*state)
    b.set_state(*state)
    ra, rb = a.pmg_cycle(4), b.pmg_cycle(4)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])
    b.set_timing(True)
    b.set_state(*state)
    rt = b.pmg_cycle(4)
    np.testing.assert_array_equal(ra, rt)
    t = b.timing()
    assert t["k_face"][1] == 4 * 2 and (t["k_sweep"][1] > 0 or t["k_lo_solve"][1] == 4)
    assert a.launch_count() >= 4 * a.launches_per_call(True)


def test_divergence_is_reported_not_trapped(libs):
    """A state with negative pressure sets the device status word; the call
    returns CGKS_EDIVERGED and the context stays usable."""
    cgks, _ = libs
    mesh, spec, state = case("cavity8")
    g = cgks.Solver(cgks.Mesh(mesh), spec)
    W = state[0].copy()
    W[3, 3] = -1.0
    g.set_state(W)
    with pytest.raises(cgks.CgksError) as e:
        g.pmg_cycle(2)
    assert e.value.status == -5
    with pytest.raises(cgks.CgksError):
        g.explicit_steps(1)
    g.set_state(*state)          # recovers
    g.pmg_cycle(1)


def test_zero_cycles_and_bad_arguments(libs):
    cgks, _ = libs
    mesh, spec, state = case("cavity8")
    g = cgks.Solver(cgks.Mesh(mesh), spec)
    g.set_state(*state)
    assert g.pmg_cycle(0).shape == (0,)
    with pytest.raises(cgks.CgksError):
        cgks.Solver(cgks.Mesh(mesh), dict(spec, bcs=[dict(kind="noslip")]))   # tag 1 has no condition


def test_cavity_2048_cells_five_cycles(libs):
    """The 2048-cell cavity workload (32 x 32 quads split in two, 10 %
    jitter, Re 1000, Ma 0.15): five V-cycles, full-field comparison."""
    mesh = MG.cavity(32)
    spec = dict(gamma=GAM, mu=0.15 / 1000, cfl_hi=0.5,
                bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(0.15, 0.0))])
    W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
    g, o = pair(libs, mesh, spec, (W, None))
    rg, ro = g.pmg_cycle(5), o.pmg_cycles(5)
    check(g, o, "cavity 2048")
    np.testing.assert_allclose(rg, ro, rtol=1e-9)


def test_cylinder_57344_cells_one_cycle(libs):
    """The full 57,344-cell hybrid cylinder O-mesh (Ma 0.38, inviscid):
    one V-cycle in the launch configuration the benchmark times."""
    mesh = MG.cylinder(256, 32, 96)
    assert mesh.n_cells == 57344
    spec = dict(gamma=GAM, mu=0.0, cfl_hi=0.4,
                bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(0.38, 0.0), p=1 / GAM)])
    W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.38, 0.0, 1 / GAM), (mesh.n_cells, 1))
    g, o = pair(libs, mesh, spec, (W, None))
    g.pmg_cycle(1)
    o.pmg_cycles(1)
    check(g, o, "cylinder 57344")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["cylinder_viscous", "mixed_slip_farfield"])
def test_fused_low_order_equals_per_phase_launches(name, precision):
    """The persistent cooperative low-order launch runs the same per-cell
    arithmetic as the per-phase kernels; the compiler may contract a few
    multiply-adds differently in the fused body (one ulp per sweep), which
    the CFL-1000 implicit solve carries along: equal to rounding (FP64), to
    the mixed path's own tolerance (FP32 sweeps)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_09965_gb300 import cgks
    mesh, spec, (W, Wx) = case(name)
    out = []
    for fused in (1, 0):
        s = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision=precision, low_order_fused=fused))
        s.set_state(W, Wx)
        h = s.pmg_cycle(4)
        out.append((s.get_state()[0], h, s.launches_per_call(True)))
    assert out[0][2] < out[1][2]
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert rel(out[0][0], out[1][0]) < tol, rel(out[0][0], out[1][0])
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=100 * tol)


def test_fused_barrier_timeout_reports_status_and_recovers():
    """A grid-barrier wait of the persistent low-order launch that runs out
    (a spin limit of one poll, so the first blocks to arrive give up) ends
    the launch early and the call returns CGKS_ETIMEOUT, not a hang.  After
    cgks_set_state and the default limit, the same solver runs V-cycles
    equal to the per-phase launches: the barrier left half-counted by the
    timed-out launch is cleared before the next one."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_09965_gb300 import cgks
    mesh, spec, (W, Wx) = case("cylinder_viscous")
    ref = cgks.Solver(cgks.Mesh(mesh), dict(spec, low_order_fused=0))
    ref.set_state(W, Wx)
    h_ref = ref.pmg_cycle(3)
    W_ref = ref.get_state()[0]
    s = cgks.Solver(cgks.Mesh(mesh), dict(spec, low_order_fused=1))
    s.set_state(W, Wx)
    s.set_barrier_spin_limit(1)
    with pytest.raises(cgks.CgksError) as e:
        s.pmg_cycle(1)
    assert e.value.status == cgks.ETIMEOUT
    s.set_barrier_spin_limit(0)
    s.set_state(W, Wx)
    h = s.pmg_cycle(3)
    assert rel(s.get_state()[0], W_ref) < 1e-13
    np.testing.assert_allclose(h, h_ref, rtol=1e-11)
    with pytest.raises(cgks.CgksError):
        s.set_barrier_spin_limit(-1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["cavity8", "mixed_slip_farfield", "cylinder_viscous"])
def test_lf_low_level_matches_oracle(libs, name, precision):
    """Lax-Friedrichs low-level flux (CGKS_FLUX_LF): V-cycles against the
    oracle's L-F variant, FP64 within 1e-12, mixed within its 1e-5."""
    mesh, spec, state = case(name)
    spec = dict(spec, flux_lo="lf")
    g, o = pair(libs, mesh, dict(spec, precision=precision), state)
    hg, ho = g.pmg_cycle(3), o.pmg_cycles(3)
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    tol = TOL if precision == "fp64" else 1e-5
    assert rel(Wg, Wo) < tol, rel(Wg, Wo)
    np.testing.assert_allclose(hg, ho, rtol=1e-9 if precision == "fp64" else 1e-3)


def test_degenerate_meshes(libs):
    """Smallest meshes against the oracle over V-cycles: two triangles (each
    cell's only neighbour is the other), and a single quad between two slip
    walls, whose rank-deficient stencil falls back to the linear
    reconstruction on both sides."""
    cgks, O = libs
    spec = dict(gamma=GAM, mu=0.01, bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(0.3, 0.1), p=1 / GAM)])
    for cells in ("tri", "quad"):
        mesh = MG.box(1, 1, cells=cells, tags=(0, 1, 0, 1))
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.3, 0.1, 1 / GAM), (mesh.n_cells, 1))
        W[0, 0] *= 1.01
        g, o = pair(libs, mesh, spec, (W, None))
        np.testing.assert_allclose(g.pmg_cycle(3), o.pmg_cycles(3), rtol=1e-9)
        check(g, o, cells)

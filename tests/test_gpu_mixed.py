"""Mixed precision (FP32 reconstruction, fluxes and sweeps; FP64
conservative variables, accumulations, residuals and diagonal inversion)
against the FP64 oracle.

Bars: per step the FP32 flux error is O(1e-7) relative; a handful of
steps stays within 1e-5 relative L2.  The converged field of a viscous
cylinder must match the FP64 converged field within 1e-6 relative L2.
The mixed residual floors where the FP32 rounding of the face fluxes
(~1e-7 relative per face) balances the correction: on this cylinder the
floor is a drop of 1.4e-6 to 2.2e-6 over the last 200 of 3000 cycles, the
same before and after the sweep's per-slot refactor (measured on GB300 at
both revisions and at the current one), so the bar is five decades, not
seven: no correction of an FP32-flux defect can fall below that floor."""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact
from tests.test_gpu_parity import case, rel

pytestmark = pytest.mark.gpu
GAM = 1.4


@pytest.fixture(scope="module")
def libs(oracle_lib):
    from paper_2109_09965_gb300 import cgks
    cgks.lib()
    return cgks, oracle_lib


@pytest.mark.parametrize("scheme", ["S1O2", "S2O4"])
@pytest.mark.parametrize("name", ["cavity8", "mixed_slip_farfield", "cylinder_inviscid", "linear_fallback"])
def test_mixed_steps_close_to_fp64_oracle(libs, name, scheme):
    cgks, O = libs
    mesh, spec, state = case(name)
    spec = dict(spec, time_scheme=scheme)
    g = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision="mixed"))
    o = O.OracleSolver(O.OracleMesh(mesh), spec)
    g.set_state(*state)
    o.set_state(*state)
    g.explicit_steps(3)
    o.explicit_steps(3)
    g.pmg_cycle(2)
    o.pmg_cycles(2)
    Wg, Xg = g.get_state()
    Wo, Xo = o.get_state()
    assert rel(Wg, Wo) < 1e-5, rel(Wg, Wo)
    assert rel(Xg, Xo) < 1e-3, rel(Xg, Xo)


def test_mixed_converged_field_matches_fp64(libs):
    """Viscous cylinder (Re 38): converge both precisions with the V-cycle."""
    cgks, _ = libs
    mesh = MG.cylinder(48, 6, 12, growth=1.15, R_far=6.0)
    ma = 0.38
    spec = dict(gamma=GAM, mu=0.01, cfl_hi=0.4,
                bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    W0 = np.tile(exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1 / GAM), (mesh.n_cells, 1))
    out = {}
    for prec in ("fp64", "mixed"):
        s = cgks.Solver(cgks.Mesh(mesh), dict(spec, precision=prec))
        s.set_state(W0)
        r = s.pmg_cycle(3000)
        out[prec] = (s.get_state()[0], r)
    W64, r64 = out["fp64"]
    W32, r32 = out["mixed"]
    assert r64[-1] < 1e-13 * r64[0] + 1e-15
    assert r32[-200:].max() < 1e-5 * r32[0]          # residual drop before the FP32 floor
    assert rel(W32, W64) < 1e-6, rel(W32, W64)

"""Pins against numbers printed in the paper (fixtures in tests/golden/)."""
import math
import os

import numpy as np

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAM = 1.4


def _rows(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_shock_reflection_states_satisfy_rankine_hugoniot(oracle_lib):
    """The two printed states of Section 4.3 sit on either side of an
    oblique shock: the oracle's Euler normal flux, and the KFVS flux of
    each state with itself, agree across the shock to the printed digits.
    The shock normal follows from continuity of the tangential velocity."""
    O = oracle_lib
    (r1, u1, v1, p1), (r2, u2, v2, p2) = [[float(x) for x in r] for r in _rows("shock_reflection_states.txt")]
    W1 = exact.cons_from_prim(GAM, r1, u1, v1, p1)
    W2 = exact.cons_from_prim(GAM, r2, u2, v2, p2)
    du = np.array([u1 - u2, v1 - v2])
    n = du / np.linalg.norm(du)
    F1, F2 = O.euler_flux(GAM, W1, n), O.euler_flux(GAM, W2, n)
    scale = np.abs(F1).max()
    assert np.abs(F1 - F2).max() < 3e-5 * scale
    spec = dict(gamma=GAM)
    K1, K2 = O.kfvs(spec, W1, W1, n), O.kfvs(spec, W2, W2, n)
    assert np.abs(K1 - K2).max() < 3e-5 * scale
    # the incident shock angle of the classic case (about 29 degrees)
    beta = math.degrees(math.atan2(-n[0], n[1]) % math.pi)
    assert 28.0 < min(beta, 180 - beta) < 30.0


def test_free_stream_has_unit_sound_speed(oracle_lib):
    O = oracle_lib
    for ma in (0.15, 0.38, 1.5):
        W = exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1.0 / GAM)
        F = O.euler_flux(GAM, W, np.array([1.0, 0.0]))
        # F = (rho u, rho u^2 + p, 0, (E + p) u) with c = sqrt(gamma p / rho) = 1
        p = F[1] - ma * ma
        assert abs(math.sqrt(GAM * p / 1.0) - 1.0) < 1e-14


def test_perturbations_do_not_grow_with_walls_and_far_field(oracle_lib):
    """Small random perturbations of a uniform flow on a jittered triangle
    mesh with slip walls, no-slip walls and a far field stay bounded: the
    boundary readings (mirror ghost cells in the reconstruction, far-field
    state from the cell mean) keep the explicit scheme stable."""
    O = oracle_lib
    mesh = MG.box(8, 8, jitter=0.1, seed=1, cells="tri", tags=(0, 1, 2, 2))
    om = O.OracleMesh(mesh)
    ma = 0.2
    spec = dict(gamma=GAM, mu=0.003, cfl_hi=0.4,
                bcs=[dict(kind="slip"), dict(kind="noslip"),
                     dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    W0 = np.tile(exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1 / GAM), (mesh.n_cells, 1))
    rng = np.random.default_rng(5)
    s = O.OracleSolver(om, spec)
    s.set_state(W0 + 1e-6 * rng.normal(size=W0.shape))
    s.explicit_steps(400)
    W, _ = s.get_state()
    # the flow adjusts to the walls (order Ma), but no mode blows up
    assert np.isfinite(W).all() and s.status() == 0
    s2 = O.OracleSolver(om, spec)
    s2.set_state(W0)
    s2.explicit_steps(400)
    Wr, _ = s2.get_state()
    assert np.abs(W - Wr).max() < 1e-4

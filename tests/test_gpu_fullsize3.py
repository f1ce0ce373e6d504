"""The 3-D configurations at full size, through the C ABI.

The oracle is too slow for a V-cycle on 512,000 or 3,072,000 cells, so at
these sizes the GPU path is checked by properties that hold at any size
(with the oracle's own geometry as the independent reference for volumes):
- a gas at rest in the closed sphere shell (no-slip sphere, slip outer
  boundary) is a steady state: V-cycles and explicit steps keep it to
  round-off (FP64 round-off in FP64, FP32 flux round-off in mixed);
- with slip walls on both boundaries no mass or energy crosses the boundary
  and interior fluxes cancel pairwise, so explicit S2O4 steps keep
  sum |Omega| rho and sum |Omega| rho E to round-off, in FP64 and in the
  mixed path (FP32 fluxes, FP64 accumulation).
The meshes are the bench's: the config-3 construction (icosphere level 4,
40 prism + 20 split-tet layers, first layer 5e-3 D) and the config-4 one
(level 5, 60 + 30 layers, first layer 1e-3 D).
"""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG

pytestmark = pytest.mark.gpu
GAM = 1.4


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_09965_gb300 import cgks
    cgks.lib()
    return cgks


def cons3(rho, u, v, w, p):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (GAM - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


SIZES = {"config3_512k": dict(level=4, n_prism=40, n_tet=20, h0=5e-3),
         "config4_3M": dict(level=5, n_prism=60, n_tet=30, h0=1e-3)}


@pytest.fixture(scope="module", params=list(SIZES))
def sphere(request, cg):
    from oracle import oracle3 as O3
    O3.build()
    mesh = MG.sphere(**SIZES[request.param])
    vol, xc, _ = O3.OracleMesh3(mesh).geometry()
    return request.param, mesh, cg.Mesh(mesh), vol, xc


def test_rest_state_is_kept(cg, sphere):
    name, mesh, gm, vol, xc = sphere
    spec = dict(gamma=GAM, mu=0.2 / 118, bcs=[dict(kind="noslip"), dict(kind="slip")])
    W0 = np.tile(cons3(1.0, 0.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
    for prec in ("fp64", "mixed"):
        s = cg.Solver(gm, dict(spec, precision=prec))
        s.set_state(W0)
        s.pmg_cycle(2)
        s.explicit_steps(1)
        W, Wx = s.get_state()
        # FP64: round-off of the closed-cell sums; mixed: FP32 face fluxes
        # (eps 6e-8) through the CFL-1000 implicit solve
        tw, tx = (1e-12, 1e-10) if prec == "fp64" else (1e-5, 1e-3)
        assert np.abs(W - W0).max() < tw * np.abs(W0).max(), (name, prec, np.abs(W - W0).max())
        assert np.abs(Wx).max() < tx, (name, prec, np.abs(Wx).max())
        s.close()


def test_closed_shell_conserves_mass_and_energy(cg, sphere):
    name, mesh, gm, vol, xc = sphere
    spec = dict(gamma=GAM, mu=0.2 / 118, time_scheme="S2O4", bcs=[dict(kind="slip"), dict(kind="slip")])
    x, y, z = xc[:, 0], xc[:, 1], xc[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    bump = 0.05 * np.exp(-((r - 1.0) ** 2))
    W0 = cons3(1.0 + bump, 0.1 * np.sin(0.3 * y), -0.05 * np.cos(0.2 * x), 0.02 * np.sin(0.1 * z),
               (1.0 + 1.4 * bump) / GAM)
    m0 = (vol[:, None] * W0).sum(0)
    for prec in ("fp64", "mixed"):
        s = cg.Solver(gm, dict(spec, precision=prec))
        s.set_state(W0)
        s.explicit_steps(2)
        W, _ = s.get_state()
        s.close()
        m1 = (vol[:, None] * W).sum(0)
        assert np.abs(W - W0).max() > 1e-6, (name, prec)            # the flow evolved
        for v in (0, 4):
            assert abs(m1[v] - m0[v]) < 1e-12 * abs(m0[v]), (name, prec, v, m1[v] - m0[v])

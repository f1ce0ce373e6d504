"""Wall loads from the GPU (cgks_wall_loads) and the force post-processing.

On a converged viscous cylinder (Re 40, Ma 0.15, the case of Section 4's
first table) the momentum fluxes through the wall and the far field balance
to the residual level, the wall face centres lie on the body, Cl vanishes by
symmetry and Cd and the separation angle fall in the ranges of the
paper's table (coarse mesh: the fine-mesh values are 1.525 and 53.3 deg)."""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from paper_2109_09965_gb300 import post
from tests import exact

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cylinder_re40_loads(cg, precision):
    ma, re, D = 0.15, 40.0, 1.0
    mesh = MG.cylinder(64, 12, 20, growth=1.1, R_far=15.0)
    spec = dict(gamma=GAM, mu=ma * D / re, precision=precision,
                bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    s = cg.Solver(cg.Mesh(mesh), spec)
    s.set_state(np.tile(exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1 / GAM), (mesh.n_cells, 1)))
    h = s.pmg_cycle(3000)
    assert h[-1] < (1e-8 if precision == "fp64" else 1e-4) * h[0], h[-1] / h[0]
    wall, far = s.wall_loads(0), s.wall_loads(1)
    assert wall["S"].size == 64 and far["S"].size == 64
    r = np.linalg.norm(wall["x"], axis=1)
    assert np.allclose(r, 0.5 * math.cos(math.pi / 64), rtol=1e-12)
    assert np.allclose(wall["n"], -wall["x"] / r[:, None], atol=1e-12)
    Fw, Ff = post.body_force(wall), post.body_force(far)
    assert np.abs(Fw + Ff).max() < 2e-3 * np.abs(Fw).max(), (Fw, Ff)
    cd, cl = post.force_coefficients(wall, rho=1.0, U=ma, ref=D)
    assert 1.3 < cd < 2.0 and abs(cl) < 0.02, (cd, cl)
    surf = post.surface_2d(wall, rho=1.0, U=ma, p_inf=1 / GAM)
    sep = post.separation_angle(surf)
    assert sep is not None and 40.0 < sep < 65.0, sep
    assert abs(surf["Cp"][0] - 1.0) < 0.3          # front stagnation


def test_sphere_loads_balance(cg):
    """3-D: wall face centres on the polyhedral sphere, the body force along
    the stream, and the wall and far-field momentum fluxes balanced after the
    V-cycles converge."""
    mesh = MG.sphere(2, 40, 20, h0=5e-3)
    vel = (0.2, 0.0, 0.0)
    spec = dict(gamma=GAM, mu=0.2 / 118, bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
    s = cg.Solver(cg.Mesh(mesh), spec)
    W = np.tile([1.0, 0.2, 0.0, 0.0, 1 / GAM / (GAM - 1) + 0.02], (mesh.n_cells, 1))
    s.set_state(W)
    h = s.pmg_cycle(1500)
    assert h[-1] < 1e-5 * h[0], h[-1] / h[0]
    wall, far = s.wall_loads(0), s.wall_loads(1)
    assert wall["S"].size > 0 and wall["x"].shape[1] == 3
    r = np.linalg.norm(wall["x"], axis=1)
    assert r.max() <= 0.5 + 1e-12 and r.min() > 0.45
    Fw, Ff = post.body_force(wall), post.body_force(far)
    assert Fw[0] > 0 and abs(Fw[1]) < 0.1 * Fw[0] and abs(Fw[2]) < 0.1 * Fw[0]
    assert np.abs(Fw + Ff).max() < 5e-3 * Fw[0], (Fw, Ff)

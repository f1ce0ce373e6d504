"""Pins of the 3-D oracle's full gas-kinetic flux (Eq. (2nd-flux)) and
compact WENO weights.

* With w = 0 and z-independent data the 3-D full flux is the 2-D oracle's
  full flux (pinned by brute-force quadrature in test_oracle_fullflux).
* Continuous data reduce it to the 3-D smooth flux for any tau_n; tau = 0
  with tau_n -> infinity gives the 3-D KFVS flux at t = 0; antisymmetry;
  rotating the whole problem rotates the result (all three slope
  directions, whatever the face frame).
* WENO: epsilon -> infinity gives the linear weights; linear fields stay
  exact for any epsilon; a front's overshoot is cut.
"""
import math

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests.test_oracle3 import GAM, O3, rand_normal, rand_state  # noqa: F401  (O3 is a fixture)


def lift(W):
    return np.array([W[0], W[1], W[2], 0.0, W[3]])


def liftg(G):
    g = np.zeros((3, 5))
    for d in range(2):
        g[d] = lift(G[d])
    return g


def test_full_flux_reduces_to_the_2d_oracle(O3, oracle_lib):
    O2 = oracle_lib
    rng = np.random.default_rng(40)
    for _ in range(5):
        spec = dict(gamma=GAM, mu=rng.uniform(0.0, 0.03), tau_c1=0.05, tau_c2=1.0)
        rho_l, rho_r = rng.uniform(0.6, 1.6, 2)
        W2l = np.array([rho_l, rho_l * 0.3, -rho_l * 0.1, 1.0 / (GAM - 1) + 0.5 * rho_l * 0.1])
        W2r = np.array([rho_r, rho_r * 0.25, rho_r * 0.05, 1.3 / (GAM - 1) + 0.5 * rho_r * 0.065])
        G2l, G2r = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
        th = rng.uniform(0, 2 * np.pi)
        n2 = np.array([math.cos(th), math.sin(th)])
        delta, dt = rng.uniform(0.05, 0.2), rng.uniform(0.002, 0.02)
        a2 = O2.gks_full_flux_point(spec, W2l, W2r, G2l, G2r, n2, delta, dt)
        a3 = O3.gks_full_flux_point(spec, lift(W2l), lift(W2r), liftg(G2l), liftg(G2r),
                                    np.array([n2[0], n2[1], 0.0]), delta, dt)
        for x2, x3 in zip(a2, a3):
            sc = max(1.0, np.abs(x2).max())
            np.testing.assert_allclose(x3[[0, 1, 2, 4]], x2, rtol=1e-10, atol=1e-12 * sc)
            assert abs(x3[3]) < 1e-12 * sc


def test_full_flux_limits_and_antisymmetry(O3):
    rng = np.random.default_rng(41)
    for _ in range(3):
        W = rand_state(rng, 0.7)
        G = rng.normal(size=(3, 5)) * 0.2
        n = rand_normal(rng)
        dt = rng.uniform(0.002, 0.03)
        spec = dict(gamma=GAM, mu=0.01, tau_c1=0.3, tau_c2=1.0)
        full = O3.gks_full_flux_point(spec, W, W, G, G, n, 0.1, dt)
        smooth = O3.gks_flux_point(spec, W, W, G, G, n, 0.1)
        for a, b in zip(full, smooth):
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-11 * max(1.0, np.abs(b).max()))
        Wl, Wr = rand_state(rng), rand_state(rng)
        z = np.zeros((3, 5))
        kf = dict(gamma=GAM, mu=0.0, tau_c1=1e9, tau_c2=0.0)
        F0, F1, _, _ = O3.gks_full_flux_point(kf, Wl, Wr, z, z, n, 0.0, 0.01)
        np.testing.assert_allclose(F0, O3.kfvs(kf, Wl, Wr, n), rtol=1e-7, atol=1e-8)
        Gl, Gr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        a = O3.gks_full_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.05, 0.02)
        b = O3.gks_full_flux_point(spec, Wr, Wl, Gr, Gl, -n, 0.05, 0.02)
        np.testing.assert_allclose(a[0], -b[0], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(a[2], b[2], rtol=1e-11, atol=1e-12)


def cell_means_linear(mesh, C):
    """Means and mean gradients of the linear field C[0] + x C[1] + y C[2] +
    z C[3]: the value at the centroid (tet decomposition from the node
    mean, as exact for linear fields) and the constant gradient."""
    W = np.zeros((mesh.n_cells, 5))
    Wx = np.zeros((mesh.n_cells, 3, 5))
    from oracle import oracle3
    om = oracle3.OracleMesh3(mesh)
    _, xc, _ = om.geometry()
    for c in range(mesh.n_cells):
        W[c] = C[0] + xc[c, 0] * C[1] + xc[c, 1] * C[2] + xc[c, 2] * C[3]
        Wx[c] = C[1:4]
    return W, Wx, om


@pytest.mark.parametrize("eps", [1e-2, 1e-6])
def test_weno3_exact_for_linear_fields(O3, eps):
    mesh = MG.box3(3, 3, 2, jitter=0.2, seed=42, cells="tet", tags=(0, 0, 0, 0, 0, 0))
    C = np.random.default_rng(43).normal(size=(4, 5)) * 0.2
    C[0] += np.array([1.5, 0.2, 0.1, 0.1, 4.0])
    W, Wx, om = cell_means_linear(mesh, C)
    s = O3.OracleSolver3(om, dict(gamma=GAM, weno_eps=eps, bcs=[dict(kind="farfield")]))
    s.set_state(W, Wx)
    s.reconstruct()
    F = om.faces()
    for k in range(om.n_faces):
        for q in range(F["ng"][k]):
            x = F["xg"][k, q]
            v, g = s.recon_eval(F["c0"][k], x)
            np.testing.assert_allclose(v, C[0] + x @ C[1:4], rtol=1e-11, atol=1e-11)
            np.testing.assert_allclose(g, C[1:4], rtol=1e-9, atol=1e-9)


def test_weno3_linear_weight_limit_and_front(O3):
    mesh = MG.box3(4, 3, 3, jitter=0.15, seed=44, cells="hex", tags=(0, 0, 0, 0, 0, 0))
    om = O3.OracleMesh3(mesh)
    _, xc, _ = om.geometry()
    s_ = np.tanh((xc[:, 0] - 0.52) / 0.02)
    W = np.stack([1.5 + 0.5 * s_, 0.2 + 0.1 * s_, 0.05 * s_, 0.0 * s_, 3.0 + s_], -1)
    Wx = np.zeros((mesh.n_cells, 3, 5))
    Wx[:, 0, :] = np.array([0.5, 0.1, 0.05, 0.0, 1.0])[None, :] * (1 - s_ ** 2)[:, None] / 0.02 * 0.25
    F = om.faces()

    def vals(spec):
        s = O3.OracleSolver3(om, spec)
        s.set_state(W, Wx)
        s.reconstruct()
        return np.array([s.recon_eval(F["c0"][k], F["xg"][k, q])[0]
                         for k in range(om.n_faces) for q in range(F["ng"][k])])
    base = dict(gamma=GAM, bcs=[dict(kind="farfield")])
    v0 = vals(base)
    np.testing.assert_allclose(vals(dict(base, weno_eps=1e30)), v0, rtol=1e-12, atol=1e-12)
    lo, hi = W.min(0), W.max(0)
    lin = np.maximum(v0 - hi, lo - v0).max()
    nl_v = vals(dict(base, weno_eps=1e-6))
    nl = np.maximum(nl_v - hi, lo - nl_v).max()
    assert lin > 0.02, lin
    assert nl < 0.5 * lin, (nl, lin)


def test_full_flux_rotation_invariance(O3):
    """Rotating the whole problem (states, gradients, normal) by a random
    rotation rotates the full flux and interface state: exercises the
    slopes along all three local axes, which the reduction to 2-D leaves
    out for the second tangent."""
    rng = np.random.default_rng(45)
    spec = dict(gamma=GAM, mu=0.01, tau_c1=0.05, tau_c2=1.0)
    for _ in range(3):
        Wl, Wr = rand_state(rng), rand_state(rng)
        Gl, Gr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        n = rand_normal(rng)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))

        def rotW(W):
            return np.concatenate([[W[0]], Q @ W[1:4], [W[4]]])

        def rotG(G):
            return Q @ np.array([rotW(G[d]) for d in range(3)])
        a = O3.gks_full_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.1, 0.01)
        b = O3.gks_full_flux_point(spec, rotW(Wl), rotW(Wr), rotG(Gl), rotG(Gr), Q @ n, 0.1, 0.01)
        for x, y in zip(a, b):
            np.testing.assert_allclose(y, rotW(x), rtol=1e-10, atol=1e-11 * max(1.0, np.abs(x).max()))

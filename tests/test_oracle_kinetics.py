"""Pins of the oracle's kinetic layer (Section 2.2 of the paper).

Every expected value here comes from outside the oracle: brute-force
quadrature of the Maxwellian in (u, v, xi^2), the Euler equations, and the
Navier-Stokes closure the paper states for the BGK model (tau = mu/p,
Pr = 1).  A dropped moment term, a wrong sign or a transposed frame in
the oracle fails one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import gamma as Gamma
from scipy.special import roots_genlaguerre

from tests import exact

GAM = 1.4
K2D = (4 - 2 * GAM) / (GAM - 1)          # internal degrees of freedom in 2-D
N_DOF = K2D + 2                           # total degrees of freedom


def brute_moments(W, f, urange=0):
    """rho * E[f(u, v, s) psi] for the Maxwellian of W (global frame), by
    Gauss-Legendre in u (truncated at 12 sigma), Gauss-Hermite in v and
    generalised Gauss-Laguerre in s = xi^2."""
    rho, mx, my, E = W
    U, V = mx / rho, my / rho
    p = (GAM - 1) * (E - 0.5 * rho * (U * U + V * V))
    lam = rho / (2 * p)
    sl = math.sqrt(lam)
    lo, hi = -12.0, 12.0
    if urange > 0:
        lo = -sl * U
    elif urange < 0:
        hi = -sl * U
    xg, wg = np.polynomial.legendre.leggauss(160)
    xs = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
    ws = 0.5 * (hi - lo) * wg * np.exp(-xs * xs) / math.sqrt(math.pi)
    u = U + xs / sl
    xh, wh = np.polynomial.hermite.hermgauss(40)
    v = V + xh / sl
    wv = wh / math.sqrt(math.pi)
    alpha = K2D / 2 - 1
    yl, wl = roots_genlaguerre(30, alpha)
    s = yl / lam
    wsx = wl / Gamma(K2D / 2)
    UU, VV, SS = np.meshgrid(u, v, s, indexing="ij")
    WW = ws[:, None, None] * wv[None, :, None] * wsx[None, None, :]
    psi = [np.ones_like(UU), UU, VV, 0.5 * (UU ** 2 + VV ** 2 + SS)]
    fv = f(UU, VV, SS)
    return np.array([rho * np.sum(WW * fv * ps) for ps in psi])


def rand_state(rng, ma=0.8):
    rho = rng.uniform(0.5, 2.0)
    p = rng.uniform(0.4, 1.5)
    c = math.sqrt(GAM * p / rho)
    u, v = rng.uniform(-ma, ma, 2) * c
    return exact.cons_from_prim(GAM, np.float64(rho), np.float64(u), np.float64(v), np.float64(p))


def prim_grads(W, G):
    """Primitive (rho, u, v, p, T) gradients from conservative W and G[d][v]."""
    rho, mx, my, E = W
    u, v = mx / rho, my / rho
    p = (GAM - 1) * (E - 0.5 * rho * (u * u + v * v))
    out = {}
    for d in range(2):
        dr, dmx, dmy, dE = G[d]
        du = (dmx - u * dr) / rho
        dv = (dmy - v * dr) / rho
        dp = (GAM - 1) * (dE - 0.5 * (u * u + v * v) * dr - rho * (u * du + v * dv))
        dT = (dp * rho - p * dr) / rho ** 2
        out[d] = (dr, du, dv, dp, dT)
    return (rho, u, v, p), out


SPEC = dict(gamma=GAM, mu=0.0)


def test_full_range_moments_match_quadrature(oracle_lib):
    """W^c of two equal states is their own conservative vector (half-range
    moments of both sides add up to the full moments)."""
    O = oracle_lib
    rng = np.random.default_rng(0)
    for _ in range(5):
        W = rand_state(rng)
        Wq = brute_moments(W, lambda u, v, s: 1.0)
        np.testing.assert_allclose(Wq, W, rtol=1e-12, atol=1e-13)
        n = np.array([1.0, 0.0])
        _, _, Wc, _ = O.gks_flux_point(SPEC, W, W, np.zeros((2, 4)), np.zeros((2, 4)), n)
        np.testing.assert_allclose(Wc, W, rtol=1e-14, atol=1e-14)


def test_half_range_equilibrium_state(oracle_lib):
    """W^c = int psi [g^l H(u_n) + g^r (1 - H(u_n))] by brute force."""
    O = oracle_lib
    rng = np.random.default_rng(1)
    for _ in range(5):
        Wl, Wr = rand_state(rng), rand_state(rng)
        n = np.array([1.0, 0.0])
        _, _, Wc, _ = O.gks_flux_point(SPEC, Wl, Wr, np.zeros((2, 4)), np.zeros((2, 4)), n)
        ref = brute_moments(Wl, lambda u, v, s: 1.0, +1) + brute_moments(Wr, lambda u, v, s: 1.0, -1)
        np.testing.assert_allclose(Wc, ref, rtol=1e-11, atol=1e-12)


def test_kfvs_matches_quadrature_and_euler(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(2)
    for _ in range(5):
        Wl, Wr = rand_state(rng), rand_state(rng)
        n = np.array([1.0, 0.0])
        F = O.kfvs(SPEC, Wl, Wr, n)
        ref = (brute_moments(Wl, lambda u, v, s: u, +1) + brute_moments(Wr, lambda u, v, s: u, -1))
        np.testing.assert_allclose(F, ref, rtol=1e-11, atol=1e-12)
        # equal states: the split fluxes add up to the Euler flux
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        np.testing.assert_allclose(O.kfvs(SPEC, Wl, Wl, n), exact.euler_flux(GAM, Wl, n),
                                   rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(O.euler_flux(GAM, Wl, n), exact.euler_flux(GAM, Wl, n),
                                   rtol=1e-14, atol=1e-15)
        # antisymmetry
        np.testing.assert_allclose(O.kfvs(SPEC, Wl, Wr, n), -O.kfvs(SPEC, Wr, Wl, -n),
                                   rtol=1e-13, atol=1e-14)


def test_micro_slope_compatibility(oracle_lib):
    """<a psi> = dW for the solved micro-slope a (Section 2.2)."""
    O = oracle_lib
    rng = np.random.default_rng(3)
    for _ in range(5):
        W = rand_state(rng)
        dW = rng.normal(size=4)
        s = O.micro_slope(GAM, W, dW)
        got = brute_moments(W, lambda u, v, x: s[0] + s[1] * u + s[2] * v + s[3] * 0.5 * (u * u + v * v + x))
        np.testing.assert_allclose(got, dW, rtol=1e-11, atol=1e-12)


def test_uniform_state_gives_euler_flux(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(4)
    spec = dict(gamma=GAM, mu=0.01)
    for _ in range(5):
        W = rand_state(rng)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        F0, F1, Wc, Wt = O.gks_flux_point(spec, W, W, np.zeros((2, 4)), np.zeros((2, 4)), n)
        np.testing.assert_allclose(F0, exact.euler_flux(GAM, W, n), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(F1, 0.0, atol=1e-14)
        np.testing.assert_allclose(Wt, 0.0, atol=1e-14)
        np.testing.assert_allclose(Wc, W, rtol=1e-14)


def complex_jacobian(W, n):
    J = np.zeros((4, 4))
    h = 1e-30
    for k in range(4):
        Wc = W.astype(complex)
        Wc[k] += 1j * h
        J[:, k] = np.imag(exact.euler_flux(GAM, Wc, n)) / h
    return J


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_chapman_enskog_navier_stokes(oracle_lib, seed):
    """For a linear field (equal side states and gradients) the smooth GKS
    flux is the Navier-Stokes flux with tau = mu/p and Pr = 1 (Section 2):
      W_t = -(A_x W_x + A_y W_y)  (Euler time derivative),
      F1  = A_n W_t,
      F0  = F_Euler.n - (0, sigma.n, u.sigma.n + kappa dT/dn),
    sigma_ij = mu (du_i/dx_j + du_j/dx_i - 2/N delta_ij div u),
    kappa = mu c_p, c_p = (N + 2)/2, N = K + 2 degrees of freedom."""
    O = oracle_lib
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.001, 0.05)
    spec = dict(gamma=GAM, mu=mu)
    W = rand_state(rng, ma=0.5)
    G = rng.normal(size=(2, 4)) * 0.3
    th = rng.uniform(0, 2 * np.pi)
    n = np.array([math.cos(th), math.sin(th)])
    F0, F1, Wc, Wt = O.gks_flux_point(spec, W, W, G, G, n)
    Jx = complex_jacobian(W, np.array([1.0, 0.0]))
    Jy = complex_jacobian(W, np.array([0.0, 1.0]))
    Jn = complex_jacobian(W, n)
    Wt_ref = -(Jx @ G[0] + Jy @ G[1])
    np.testing.assert_allclose(Wc, W, rtol=1e-14)
    np.testing.assert_allclose(Wt, Wt_ref, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(F1, Jn @ Wt_ref, rtol=1e-11, atol=1e-12)
    (rho, u, v, p), dg = prim_grads(W, G)
    du = np.array([[dg[0][1], dg[1][1]], [dg[0][2], dg[1][2]]])   # du[i][j] = d u_i / d x_j
    div = du[0, 0] + du[1, 1]
    sigma = mu * (du + du.T - 2.0 / N_DOF * div * np.eye(2))
    gradT = np.array([dg[0][4], dg[1][4]])
    kappa = mu * (N_DOF + 2) / 2
    sn = sigma @ n
    visc = np.array([0.0, sn[0], sn[1], u * sn[0] + v * sn[1] + kappa * gradT @ n])
    ref = exact.euler_flux(GAM, W, n) - visc
    np.testing.assert_allclose(F0, ref, rtol=1e-11, atol=1e-12)


def test_flux_rotation_and_antisymmetry(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(8)
    spec = dict(gamma=GAM, mu=0.02)
    Wl, Wr = rand_state(rng), rand_state(rng)
    gl, gr = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
    n = np.array([0.6, 0.8])
    F0, F1, Wc, Wt = O.gks_flux_point(spec, Wl, Wr, gl, gr, n)
    # swapping sides and flipping the normal reverses the flux
    G0, G1, Vc, Vt = O.gks_flux_point(spec, Wr, Wl, gr, gl, -n)
    np.testing.assert_allclose(G0, -F0, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G1, -F1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Vc, Wc, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Vt, Wt, rtol=1e-12, atol=1e-13)
    # rotating the whole problem rotates the flux
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])

    def rotW(W):
        out = W.copy()
        out[1:3] = R @ W[1:3]
        return out

    def rotG(G):
        # gradient of the rotated field at the rotated point: R G R^T on momentum,
        # R G on scalars
        Gr = np.zeros_like(G)
        for v in (0, 3):
            Gr[:, v] = R @ G[:, v]
        Jm = np.array([[G[0, 1], G[1, 1]], [G[0, 2], G[1, 2]]])   # Jm[a][b] = d m_a / d x_b
        Jr = R @ Jm @ R.T
        Gr[0, 1], Gr[1, 1], Gr[0, 2], Gr[1, 2] = Jr[0, 0], Jr[0, 1], Jr[1, 0], Jr[1, 1]
        return Gr

    H0, H1, Hc, Ht = O.gks_flux_point(spec, rotW(Wl), rotW(Wr), rotG(gl), rotG(gr), R @ n)
    np.testing.assert_allclose(H0, rotW(F0), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(H1, rotW(F1), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Ht, rotW(Wt), rtol=1e-12, atol=1e-13)


def test_wall_ghost_states(oracle_lib):
    """Slip wall: no mass or energy flux, W^c has zero normal velocity.
    No-slip wall: W^c moves with the wall; mass flux zero."""
    O = oracle_lib
    rng = np.random.default_rng(9)
    uw = np.array([0.3, -0.1])
    n = np.array([0.8, -0.6])
    t = np.array([-n[1], n[0]])
    uw_t = (uw @ t) * t                         # wall moves tangentially
    spec = dict(gamma=GAM, mu=0.01, bcs=[dict(kind="slip"), dict(kind="noslip", uw=tuple(uw_t))])
    for _ in range(4):
        W = rand_state(rng, 0.5)
        G = rng.normal(size=(2, 4)) * 0.2
        Wg, Gg = O.ghost(spec, 0, W, G, n)
        F0, F1, Wc, Wt = O.gks_flux_point(spec, W, Wg, G, Gg, n)
        assert abs(Wc[1] * n[0] + Wc[2] * n[1]) < 1e-14
        assert abs(F0[0]) < 1e-14 and abs(F1[0]) < 1e-14 and abs(F0[3]) < 1e-13
        Wg, Gg = O.ghost(spec, 1, W, G, n)
        F0, F1, Wc, Wt = O.gks_flux_point(spec, W, Wg, G, Gg, n)
        np.testing.assert_allclose(Wc[1:3] / Wc[0], uw_t, atol=1e-14)
        assert abs(F0[0]) < 1e-14


def test_farfield_ghost_is_free_stream(oracle_lib):
    O = oracle_lib
    ma = 0.38
    spec = dict(gamma=GAM, bcs=[dict(kind="farfield", rho=1.0, u=(ma, 0.0), p=1 / GAM)])
    W = exact.cons_from_prim(GAM, 1.0, ma, 0.0, 1 / GAM)
    for th in np.linspace(0, 2 * np.pi, 7):
        n = np.array([math.cos(th), math.sin(th)])
        Wg, _ = O.ghost(spec, 0, W, np.zeros((2, 4)), n)
        np.testing.assert_allclose(Wg, W, rtol=1e-14, atol=1e-15)

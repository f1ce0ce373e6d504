"""Pins of the oracle's full gas-kinetic flux, Eq. (2nd-flux) of the paper.

The expected values come from outside the oracle's own arithmetic:
- brute-force quadrature in velocity space (Gauss-Legendre / Hermite /
  Laguerre) and in time (Gauss-Legendre on [0, T]) of the distribution of
  Eq. (2nd-flux), written out here from the paper with the micro-slopes
  solved from brute-force moments;
- the reduction the paper states: for continuous data (g^l = g^r = g^c,
  equal slopes) Eq. (2nd-flux) collapses to Eq. (2nd-smooth-flux) whatever
  tau_n is (the smooth flux is pinned in test_oracle_kinetics);
- the two limits of the numerical collision time: tau_n -> 0 (Euler, no
  free-transport part: the smooth flux with tau = 0) and tau_n -> infinity
  (pure free transport at t = 0: the KFVS flux of the two side states,
  pinned by quadrature in test_oracle_kinetics);
- antisymmetry under swapping the sides and reversing the normal.
A dropped term, a swapped Heaviside side or a wrong time integral fails
one of them.
"""
import math

import numpy as np
import pytest

from tests.test_oracle_kinetics import GAM, brute_moments, rand_state

N = np.array([1.0, 0.0])


def slopes_brute(O, W, dn, dt):
    """a_n, a_t from the oracle's pinned micro-slope solve, A from the
    compatibility condition <(a_n u + a_t v + A) psi> = 0 with brute-force
    moments."""
    an = O.micro_slope(GAM, W, dn)
    at = O.micro_slope(GAM, W, dt)
    rhs = -brute_moments(W, lambda u, v, s: lin(an, u, v, s) * u + lin(at, u, v, s) * v)
    return an, at, O.micro_slope(GAM, W, rhs)


def lin(a, u, v, s):
    return a[0] + a[1] * u + a[2] * v + a[3] * 0.5 * (u * u + v * v + s)


def brute_full(O, spec, Wl, Wr, Gl, Gr, delta, T):
    """Fhat(T) = int_0^T <u psi f> dt and W_p(t) = <psi f(t)> at t = T/2, T,
    for n = (1, 0) (local frame = global frame), by quadrature."""
    mu, c1, c2, alpha = spec["mu"], spec.get("tau_c1", 0.01), spec.get("tau_c2", 1.0), spec.get("alpha", 0.5)
    # equilibrium state by half-range quadrature
    Wc = brute_moments(Wl, lambda u, v, s: 1.0, +1) + brute_moments(Wr, lambda u, v, s: 1.0, -1)
    dWn = 0.5 * (Gl[0] + Gr[0]) + (alpha * (Wr - Wl) / delta if delta > 0 else 0.0)
    dWt = 0.5 * (Gl[1] + Gr[1])
    anc, atc, Ac = slopes_brute(O, Wc, dWn, dWt)
    anl, atl, Al = slopes_brute(O, Wl, Gl[0], Gl[1])
    anr, atr, Ar = slopes_brute(O, Wr, Gr[0], Gr[1])

    def pres(W):
        return (GAM - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])

    tau = mu / pres(Wc)
    pl, pr = pres(Wl), pres(Wr)
    taun = tau + c1 * T + c2 * T * abs(pl - pr) / (pl + pr)

    def coefs(t):
        e = math.exp(-t / taun)
        return 1 - e, (t + tau) * e - tau, t - tau + tau * e, e

    # velocity moments of every piece, with weight w(u) = 1 (state) or u (flux)
    def pieces(wfun):
        c0 = brute_moments(Wc, lambda u, v, s: wfun(u))
        c1_ = brute_moments(Wc, lambda u, v, s: wfun(u) * (lin(anc, u, v, s) * u + lin(atc, u, v, s) * v))
        c2_ = brute_moments(Wc, lambda u, v, s: wfun(u) * lin(Ac, u, v, s))
        side = []
        for W, an, at, A, rng in ((Wl, anl, atl, Al, +1), (Wr, anr, atr, Ar, -1)):
            base = brute_moments(W, lambda u, v, s: wfun(u) * (1 - tau * (lin(an, u, v, s) * u + lin(at, u, v, s) * v)
                                                             - tau * lin(A, u, v, s)), rng)
            adv = brute_moments(W, lambda u, v, s: wfun(u) * (lin(an, u, v, s) * u + lin(at, u, v, s) * v), rng)
            side.append((base, adv))
        return c0, c1_, c2_, side

    def combine(pc, t):
        a, b, c, e = coefs(t)
        c0, c1_, c2_, side = pc
        return a * c0 + b * c1_ + c * c2_ + e * (side[0][0] + side[1][0]) - t * e * (side[0][1] + side[1][1])

    pf = pieces(lambda u: u)
    ps = pieces(lambda u: 1.0)
    xg, wg = np.polynomial.legendre.leggauss(40)

    def fhat(Tq):
        return sum(0.5 * Tq * w * combine(pf, 0.5 * Tq * (x + 1)) for x, w in zip(xg, wg))

    return fhat(T), fhat(0.5 * T), combine(ps, T), combine(ps, 0.5 * T)


@pytest.mark.parametrize("seed", [11, 12])
def test_full_flux_matches_brute_force(oracle_lib, seed):
    O = oracle_lib
    rng = np.random.default_rng(seed)
    spec = dict(gamma=GAM, mu=rng.uniform(0.002, 0.02), tau_c1=0.05, tau_c2=1.0, flux_hi="full")
    Wl, Wr = rand_state(rng, 0.6), rand_state(rng, 0.6)
    Gl, Gr = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
    delta, T = 0.05, rng.uniform(0.005, 0.03)
    F0, F1, Wc, Wt = O.gks_full_flux_point(spec, Wl, Wr, Gl, Gr, N, delta, T)
    Fd, Fh, Wd, Wh = brute_full(O, spec, Wl, Wr, Gl, Gr, delta, T)
    scale = np.abs(Fd).max()
    np.testing.assert_allclose(F0 * T + 0.5 * T * T * F1, Fd, rtol=1e-9, atol=1e-10 * scale)
    np.testing.assert_allclose(0.5 * F0 * T + 0.125 * T * T * F1, Fh, rtol=1e-9, atol=1e-10 * scale)
    np.testing.assert_allclose(Wc + T * Wt, Wd, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(Wc + 0.5 * T * Wt, Wh, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("c1", [0.0, 0.3, 50.0])
def test_continuous_data_reduces_to_smooth_flux(oracle_lib, c1):
    """g^l = g^r and equal slopes: Eq. (2nd-flux) = Eq. (2nd-smooth-flux)."""
    O = oracle_lib
    rng = np.random.default_rng(20)
    spec = dict(gamma=GAM, mu=0.01, tau_c1=c1, tau_c2=1.0)
    for _ in range(3):
        W = rand_state(rng, 0.7)
        G = rng.normal(size=(2, 4)) * 0.3
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        T = rng.uniform(0.001, 0.05)
        full = O.gks_full_flux_point(spec, W, W, G, G, n, 0.1, T)
        smooth = O.gks_flux_point(spec, W, W, G, G, n, 0.1)
        for a, b in zip(full, smooth):
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-11 * max(1.0, np.abs(b).max()))


def test_vanishing_collision_time_gives_smooth_euler_flux(oracle_lib):
    """tau = tau_n = 0: f = g^c + (a^c.u + A^c) g^c t, the smooth flux of an
    inviscid gas, for unequal side states too."""
    O = oracle_lib
    rng = np.random.default_rng(21)
    spec = dict(gamma=GAM, mu=0.0, tau_c1=0.0, tau_c2=0.0)
    for _ in range(3):
        Wl, Wr = rand_state(rng), rand_state(rng)
        Gl, Gr = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        full = O.gks_full_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.07, 0.02)
        smooth = O.gks_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.07)
        for a, b in zip(full, smooth):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13 * max(1.0, np.abs(b).max()))


def test_long_collision_time_gives_kfvs_at_t0(oracle_lib):
    """tau = 0, tau_n >> dt, uniform sides: free transport of g^l (u > 0)
    and g^r (u < 0), i.e. the KFVS flux, constant in time."""
    O = oracle_lib
    rng = np.random.default_rng(22)
    spec = dict(gamma=GAM, mu=0.0, tau_c1=1e9, tau_c2=0.0)
    z = np.zeros((2, 4))
    for _ in range(3):
        Wl, Wr = rand_state(rng), rand_state(rng)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        F0, F1, Wc, Wt = O.gks_full_flux_point(spec, Wl, Wr, z, z, n, 0.0, 0.01)
        Fk = O.kfvs(spec, Wl, Wr, n)
        np.testing.assert_allclose(F0, Fk, rtol=1e-7, atol=1e-8)
        np.testing.assert_allclose(F1, 0.0, atol=1e-5)
        _, _, Wc_s, _ = O.gks_flux_point(spec, Wl, Wr, z, z, n, 0.0)
        np.testing.assert_allclose(Wc, Wc_s, rtol=1e-7, atol=1e-8)


def test_full_flux_antisymmetry(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(23)
    spec = dict(gamma=GAM, mu=0.005, tau_c1=0.01, tau_c2=1.0)
    for _ in range(3):
        Wl, Wr = rand_state(rng), rand_state(rng)
        Gl, Gr = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([math.cos(th), math.sin(th)])
        a = O.gks_full_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.05, 0.02)
        b = O.gks_full_flux_point(spec, Wr, Wl, Gr, Gl, -n, 0.05, 0.02)
        np.testing.assert_allclose(a[0], -b[0], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(a[1], -b[1], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(a[2], b[2], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(a[3], b[3], rtol=1e-11, atol=1e-11)

"""Force and surface post-processing on synthetic wall loads (CPU)."""
import math

import numpy as np

from paper_2109_09965_gb300 import post


def circle_loads(n=360, R=0.5, p=lambda th: 0 * th, tau=lambda th: 0 * th):
    """Loads of an n-gon approximating a circle: face centres, normals out of
    the fluid (into the body), lengths, traction = p n + tau t."""
    a = (np.arange(n) + 0.5) * 2 * math.pi / n
    x = np.stack([R * np.cos(a), R * np.sin(a)], 1) * math.cos(math.pi / n)
    nrm = -np.stack([np.cos(a), np.sin(a)], 1)
    S = np.full(n, 2 * R * math.sin(math.pi / n))
    th = np.arctan2(x[:, 1], -x[:, 0]) % (2 * math.pi)
    t = np.stack([-nrm[:, 1], nrm[:, 0]], 1)
    trac = p(th)[:, None] * nrm + tau(th)[:, None] * t
    return dict(x=x, n=nrm, S=S, traction=trac)


def test_uniform_pressure_gives_no_force():
    L = circle_loads(p=lambda th: 0 * th + 3.7)
    assert np.abs(post.body_force(L)).max() < 1e-12


def test_pressure_drag_of_a_cosine_distribution():
    """p = p0 + c cos(theta) (theta from the front) pushes the body
    downstream with force c * pi * R (per unit span)."""
    R, c = 0.5, 0.8
    L = circle_loads(n=2000, R=R, p=lambda th: 1.0 + c * np.cos(th))
    F = post.body_force(L)
    assert abs(F[0] - c * math.pi * R) < 1e-5 and abs(F[1]) < 1e-9
    cd, cl = post.force_coefficients(L, rho=1.0, U=2.0, ref=2 * R)
    assert abs(cd - c * math.pi * R / (0.5 * 4.0 * 2 * R)) < 1e-5 and abs(cl) < 1e-9
    s = post.surface_2d(L, rho=1.0, U=2.0, p_inf=1.0)
    assert np.allclose(s["Cp"], c * np.cos(np.radians(s["theta"])) / 2.0, atol=1e-12)


def test_separation_angle_from_the_shear_sign_change():
    """Shear positive from the front stagnation point to 130 deg, negative
    behind it: separation 50 deg from the rear."""
    L = circle_loads(n=720, tau=lambda th: np.sin(th) * (np.radians(130.0) - np.where(th > np.pi, 2 * np.pi - th, th)))
    s = post.surface_2d(L, rho=1.0, U=1.0, p_inf=0.0)
    assert abs(post.separation_angle(s) - 50.0) < 0.1


def test_wake_length_from_the_axis_velocity():
    x = np.linspace(0.55, 5.0, 200)
    xc = np.stack([x, np.zeros_like(x)], 1)
    u = np.where(x < 0.5 + 2.2, -0.1, 0.2)              # recirculation up to 2.2 D behind the rear
    W = np.stack([np.ones_like(x), u, 0 * x, 0 * x + 2.5], 1)
    L = post.wake_length(xc, W, R=0.5, D=1.0, band=0.01)
    assert abs(L - 2.2) < 0.03


def test_shock_standoff_from_the_axis_density():
    """A bow shock 0.3 D in front of a sphere of radius 0.5: density from 1
    up to the normal-shock ratio at Ma 1.5 (1.862) over a thin tanh, then
    the stagnation rise; scattered cells around the upstream axis."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-3.0, -0.51, 4000)
    yz = rng.normal(size=(4000, 2)) * 0.02
    xc = np.column_stack([x, yz])
    ratio = 2.4 * 2.25 / (0.4 * 2.25 + 2.0)
    xs = -0.5 - 0.3
    rho = 1.0 + (ratio - 1.0) * 0.5 * (1.0 + np.tanh((x - xs) / 0.01)) + 0.1 * np.clip(x - xs, 0.0, None)
    W = np.column_stack([rho, 1.5 * rho, 0 * x, 0 * x, 2.5 + 0 * x])
    d = post.shock_standoff(xc, W, R=0.5, D=1.0, mach=1.5, angle_band=0.1)
    assert abs(d - 0.3) < 0.01, d
    d2 = post.shock_standoff(xc, W, R=0.5, D=1.0, mach=1.5, band=0.05)
    assert abs(d2 - 0.3) < 0.01, d2
    # subsonic-like field without a jump: no shock found
    assert post.shock_standoff(xc, np.column_stack([1 + 0 * x, 0 * x, 0 * x, 0 * x, 2.5 + 0 * x]), R=0.5, D=1.0,
                               mach=1.5, band=0.05) is None


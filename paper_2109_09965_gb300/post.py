"""Force and surface quantities of a converged field (Section 4's tables).

Inputs are the wall loads the library evaluates on the GPU
(`Solver.wall_loads(tag)`: per boundary face its centre, unit normal out of
the fluid, length / area and the momentum flux the fluid exerts there) and,
for the wake, the cell states.  Definitions:
  Cp = (p - p_inf) / (rho_inf U_inf^2 / 2),  p = traction . n
  Cf = tau / (rho_inf U_inf^2 / 2),  tau = traction . t (2-D: t the
       surface tangent in the direction of increasing theta, which runs
       from the front stagnation point to the rear over the upper surface)
  Cd, Cl = force along / across the free stream / (q_inf * reference)
with the reference D (2-D, per unit span) or pi D^2 / 4 (3-D).
Shock stand-off (supersonic bodies): distance from the front of the body
to the bow shock on the upstream axis, in units of D.
"""
from __future__ import annotations

import math

import numpy as np


def body_force(loads: dict) -> np.ndarray:
    """Force of the fluid on the boundary: sum over faces of S * traction."""
    return (loads["S"][:, None] * loads["traction"]).sum(0)


def force_coefficients(loads: dict, rho: float, U: float, ref: float, aoa: float = 0.0) -> tuple[float, float]:
    """(Cd, Cl) for a free stream at angle of attack aoa (radians) in the x-y
    plane; ref = D in 2-D, the frontal area in 3-D."""
    F = body_force(loads)
    q = 0.5 * rho * U * U
    drag = F[0] * math.cos(aoa) + F[1] * math.sin(aoa)
    lift = -F[0] * math.sin(aoa) + F[1] * math.cos(aoa)
    return drag / (q * ref), lift / (q * ref)


def surface_2d(loads: dict, rho: float, U: float, p_inf: float, centre=(0.0, 0.0)) -> dict:
    """Per wall face of a 2-D body: angle theta (degrees) from the front
    stagnation point (upstream, -x), increasing over the upper surface
    (y > 0) towards the rear (180) and on round the lower one; Cp and Cf,
    sorted by theta."""
    x = loads["x"] - np.asarray(centre)
    n = loads["n"]
    t = loads["traction"]
    q = 0.5 * rho * U * U
    p = (t * n).sum(1)
    tang = np.stack([-n[:, 1], n[:, 0]], 1)          # n points into the body; this is the +theta tangent
    tau = (t * tang).sum(1)
    theta = np.degrees(np.arctan2(x[:, 1], -x[:, 0])) % 360.0
    order = np.argsort(theta)
    return dict(theta=theta[order], Cp=(p[order] - p_inf) / q, Cf=tau[order] / q)


def separation_angle(surf: dict) -> float | None:
    """Separation angle measured from the rear stagnation point (degrees), on
    the upper surface: where the wall shear changes sign between the front
    stagnation point and the rear (linear interpolation)."""
    th, cf = surf["theta"], surf["Cf"]
    upper = (th > 1.0) & (th < 179.0)
    th, cf = th[upper], cf[upper]
    s = np.sign(cf)
    k = np.nonzero(s[1:] != s[:-1])[0]
    if k.size == 0:
        return None
    k = k[-1]                                         # the last change before the rear
    a = th[k] + (th[k + 1] - th[k]) * cf[k] / (cf[k] - cf[k + 1])
    return 180.0 - a


def wake_length(xc: np.ndarray, W: np.ndarray, R: float, D: float, band: float | None = None,
                angle_band: float | None = None) -> float | None:
    """Length of the recirculation behind a body centred at the origin in a
    stream along +x, from its rear surface, in units of D: the streamwise
    velocity of the cells near the downstream axis changes sign downstream
    of x = R.  Near the axis: |y| (and |z| in 3-D) < band, or, for O-meshes,
    the polar angle from the +x axis < angle_band (radians)."""
    u = W[:, 1] / W[:, 0]
    near = xc[:, 0] > R
    if angle_band is not None:
        off = np.sqrt((xc[:, 1:] ** 2).sum(1))
        near &= np.arctan2(off, xc[:, 0]) < angle_band
    else:
        near &= np.abs(xc[:, 1]) < band
        if xc.shape[1] == 3:
            near &= np.abs(xc[:, 2]) < band
    if not near.any():
        return None
    x, v = xc[near, 0], u[near]
    order = np.argsort(x)
    x, v = x[order], v[order]
    neg = np.nonzero(v < 0.0)[0]
    if neg.size == 0:
        return 0.0
    k = neg[-1]
    if k + 1 >= x.size:
        return None
    xe = x[k] + (x[k + 1] - x[k]) * (-v[k]) / (v[k + 1] - v[k])
    return (xe - R) / D


def shock_standoff(xc: np.ndarray, W: np.ndarray, R: float, D: float, mach: float, gamma: float = 1.4,
                   rho_inf: float = 1.0, band: float | None = None, angle_band: float | None = None) -> float | None:
    """Bow-shock stand-off distance in front of a body centred at the
    origin in a stream along +x, in units of D: on the upstream axis (cells
    with x < -R and |y| (|z|) < band, or polar angle from the -x axis below
    angle_band), the shock is where the density coming from upstream first
    reaches the mean of the free-stream density and the density behind a
    normal shock at the free-stream Mach number,
    rho_2 / rho_1 = (gamma + 1) M^2 / ((gamma - 1) M^2 + 2)
    (linear interpolation between the two cells around it); the stand-off
    is the distance from there to the body's front point x = -R."""
    x = xc[:, 0]
    near = x < -R
    if angle_band is not None:
        off = np.sqrt((xc[:, 1:] ** 2).sum(1))
        near &= np.arctan2(off, -x) < angle_band
    else:
        near &= np.abs(xc[:, 1]) < band
        if xc.shape[1] == 3:
            near &= np.abs(xc[:, 2]) < band
    if not near.any():
        return None
    xs, rho = x[near], W[near, 0]
    order = np.argsort(xs)
    xs, rho = xs[order], rho[order]
    m2 = mach * mach
    level = rho_inf * 0.5 * (1.0 + (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0))
    above = np.nonzero(rho >= level)[0]
    if above.size == 0 or above[0] == 0:
        return None
    k = above[0]
    xk = xs[k - 1] + (xs[k] - xs[k - 1]) * (level - rho[k - 1]) / (rho[k] - rho[k - 1])
    return (-R - xk) / D


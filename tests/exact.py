"""Exact fields and test-side quadrature used to pin the oracle.

Independent of the oracle: cell averages and cell-averaged gradients are
computed here with a degree-5 triangle rule and 5-point Gauss-Legendre on
edges, and the Euler / Navier-Stokes closed forms are written from the
equations, not from the kinetic moments.
"""
import numpy as np

# Dunavant degree-5 rule on the reference triangle (barycentric, weights sum to 1)
_A1, _B1 = 0.059715871789770, 0.470142064105115
_A2, _B2 = 0.797426985353087, 0.101286507323456
BARY5 = np.array([[1 / 3, 1 / 3, 1 / 3], [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
                  [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
W5 = np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3)
_GLX, _GLW = np.polynomial.legendre.leggauss(5)
GLX, GLW = 0.5 * (_GLX + 1.0), 0.5 * _GLW


def tri_area(p0, p1, p2):
    e1, e2 = p1 - p0, p2 - p0
    return 0.5 * (e1[0] * e2[1] - e1[1] * e2[0])


def cell_averages(mesh, field):
    """Cell averages and cell-averaged gradients of ``field(x, y) -> [..., nv]``.

    Gradient averages use the divergence theorem on the polygon boundary.
    """
    nv = field(np.zeros(1), np.zeros(1)).shape[-1]
    W = np.zeros((mesh.n_cells, nv))
    Wx = np.zeros((mesh.n_cells, 2, nv))
    for c, nodes in enumerate(mesh.cells()):
        P = mesh.nodes[nodes]
        A = 0.0
        acc = np.zeros(nv)
        for k in range(1, len(P) - 1):
            tri = np.array([P[0], P[k], P[k + 1]])
            a = tri_area(*tri)
            pts = BARY5 @ tri
            acc += a * (W5[:, None] * field(pts[:, 0], pts[:, 1])).sum(0)
            A += a
        W[c] = acc / A
        g = np.zeros((2, nv))
        for k in range(len(P)):
            pa, pb = P[k], P[(k + 1) % len(P)]
            d = pb - pa
            L = np.hypot(d[0], d[1])
            nrm = np.array([d[1], -d[0]]) / L
            pts = pa[None, :] + GLX[:, None] * d[None, :]
            g += L * nrm[:, None] * (GLW[:, None] * field(pts[:, 0], pts[:, 1])).sum(0)[None, :]
        Wx[c] = g / A
    return W, Wx


def cons_from_prim(gamma, rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], -1)


def euler_flux(gamma, W, n):
    rho, mx, my, E = W
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    un = u * n[0] + v * n[1]
    return np.array([rho * un, mx * un + p * n[0], my * un + p * n[1], (E + p) * un])


def euler_jacobian(gamma, W, n, h=1e-6):
    """Central finite-difference Jacobian of the Euler normal flux."""
    J = np.zeros((4, 4))
    for k in range(4):
        d = np.zeros(4)
        d[k] = h * max(1.0, abs(W[k]))
        J[:, k] = (euler_flux(gamma, W + d, n) - euler_flux(gamma, W - d, n)) / (2 * d[k])
    return J


def isentropic_vortex(gamma, eps=5.0, U0=(1.0, 0.0), t=0.0):
    """Exact isentropic vortex translating with U0 (T_inf = rho_inf = 1)."""
    def f(x, y):
        xr, yr = x - U0[0] * t, y - U0[1] * t
        r2 = xr * xr + yr * yr
        du = eps / (2 * np.pi) * np.exp(0.5 * (1 - r2))
        T = 1 - (gamma - 1) * eps ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
        rho = T ** (1 / (gamma - 1))
        return cons_from_prim(gamma, rho, U0[0] - du * yr, U0[1] + du * xr, rho * T)
    return f

"""Pins of the 3-D oracle (Sections 2-3 of the paper in 3-D).

Expected values come from outside the 3-D oracle:
- the independently written 2-D oracle: with w = 0 and no z-dependence the
  3-D BGK model with K3 internal degrees of freedom is the 2-D model with
  K3 + 1, so the two fluxes must agree;
- brute-force quadrature of the Maxwellian in (u, v, w, xi^2);
- the Euler and Navier-Stokes closed forms;
- geometry from the raw node arrays (Keast quadrature on tets, edge-midpoint
  rule on triangles), a Python restatement of the sweep ordering;
- complex-step Jacobians of the Euler flux for the low-order level.
"""
import math
from collections import defaultdict, deque

import numpy as np
import pytest
from scipy.special import gamma as Gamma
from scipy.special import roots_genlaguerre

from paper_2109_09965_gb300 import meshgen as MG

GAM = 1.4
K3 = (5 - 3 * GAM) / (GAM - 1)
N_DOF = K3 + 3


@pytest.fixture(scope="module")
def O3():
    from oracle import oracle3
    oracle3.build()
    return oracle3


def cons3(rho, u, v, w, p):
    return np.array([rho, rho * u, rho * v, rho * w, p / (GAM - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def euler3(W, n):
    rho = W[0]
    u = W[1:4] / rho
    p = (GAM - 1) * (W[4] - 0.5 * rho * (u @ u))
    un = u @ n
    return np.concatenate([[rho * un], W[1:4] * un + p * n, [(W[4] + p) * un]])


def rand_state(rng, ma=0.8):
    rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.4, 1.5)
    c = math.sqrt(GAM * p / rho)
    u = rng.uniform(-ma, ma, 3) * c / math.sqrt(3)
    return cons3(rho, *u, p)


def rand_normal(rng):
    n = rng.normal(size=3)
    return n / np.linalg.norm(n)


SPEC = dict(gamma=GAM, mu=0.0)


# ---------------------------------------------------------------- kinetics
def brute3(W, f, urange=0):
    """rho * E[f(u, v, w, s) psi] for the Maxwellian of W: Gauss-Legendre in
    u (x-axis is the normal), Gauss-Hermite in v, w, generalised
    Gauss-Laguerre in s = xi^2 with K3 degrees of freedom."""
    rho = W[0]
    U, V, Wv = W[1:4] / rho
    p = (GAM - 1) * (W[4] - 0.5 * rho * (U * U + V * V + Wv * Wv))
    lam = rho / (2 * p)
    sl = math.sqrt(lam)
    lo, hi = -12.0, 12.0
    if urange > 0:
        lo = -sl * U
    elif urange < 0:
        hi = -sl * U
    xg, wg = np.polynomial.legendre.leggauss(120)
    xs = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
    ws = 0.5 * (hi - lo) * wg * np.exp(-xs * xs) / math.sqrt(math.pi)
    u = U + xs / sl
    xh, wh = np.polynomial.hermite.hermgauss(24)
    v, w = V + xh / sl, Wv + xh / sl
    wv = wh / math.sqrt(math.pi)
    yl, wl = roots_genlaguerre(16, K3 / 2 - 1)
    s = yl / lam
    wsx = wl / Gamma(K3 / 2)
    UU, VV, WW, SS = np.meshgrid(u, v, w, s, indexing="ij")
    WT = ws[:, None, None, None] * wv[None, :, None, None] * wv[None, None, :, None] * wsx[None, None, None, :]
    psi = [np.ones_like(UU), UU, VV, WW, 0.5 * (UU ** 2 + VV ** 2 + WW ** 2 + SS)]
    fv = f(UU, VV, WW, SS)
    return np.array([rho * np.sum(WT * fv * ps) for ps in psi])


def test_equilibrium_kfvs_and_slopes_match_quadrature(O3):
    rng = np.random.default_rng(0)
    ex = np.array([1.0, 0.0, 0.0])
    z = np.zeros((3, 5))
    for _ in range(3):
        Wl, Wr = rand_state(rng), rand_state(rng)
        np.testing.assert_allclose(brute3(Wl, lambda u, v, w, s: 1.0), Wl, rtol=1e-12, atol=1e-13)
        _, _, Wc, _ = O3.gks_flux_point(SPEC, Wl, Wr, z, z, ex)
        ref = brute3(Wl, lambda u, v, w, s: 1.0, +1) + brute3(Wr, lambda u, v, w, s: 1.0, -1)
        np.testing.assert_allclose(Wc, ref, rtol=1e-11, atol=1e-12)
        F = O3.kfvs(SPEC, Wl, Wr, ex)
        ref = brute3(Wl, lambda u, v, w, s: u, +1) + brute3(Wr, lambda u, v, w, s: u, -1)
        np.testing.assert_allclose(F, ref, rtol=1e-11, atol=1e-12)
        dW = rng.normal(size=5)
        a = O3.micro_slope(GAM, Wl, dW)
        got = brute3(Wl, lambda u, v, w, s: a[0] + a[1] * u + a[2] * v + a[3] * w
                     + a[4] * 0.5 * (u * u + v * v + w * w + s))
        np.testing.assert_allclose(got, dW, rtol=1e-11, atol=1e-12)


def test_kfvs_and_euler_identities(O3):
    rng = np.random.default_rng(1)
    for _ in range(5):
        Wl, Wr = rand_state(rng), rand_state(rng)
        n = rand_normal(rng)
        np.testing.assert_allclose(O3.kfvs(SPEC, Wl, Wl, n), euler3(Wl, n), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(O3.euler_flux(GAM, Wl, n), euler3(Wl, n), rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(O3.kfvs(SPEC, Wl, Wr, n), -O3.kfvs(SPEC, Wr, Wl, -n), rtol=1e-13, atol=1e-14)


def test_flux_reduces_to_the_2d_oracle(O3, oracle_lib):
    """w = 0 and z-independent data: the 3-D smooth flux, interface state and
    its time derivative equal the 2-D oracle's, and carry no z-momentum."""
    O2 = oracle_lib
    rng = np.random.default_rng(2)
    for _ in range(6):
        mu = rng.uniform(0.0, 0.05)
        spec = dict(gamma=GAM, mu=mu, alpha=0.5)
        rho_l, rho_r = rng.uniform(0.6, 1.6, 2)
        W2l = np.array([rho_l, rho_l * 0.3, -rho_l * 0.1, 1.0 / (GAM - 1) + 0.5 * rho_l * 0.1])
        W2r = np.array([rho_r, rho_r * 0.25, rho_r * 0.05, 1.1 / (GAM - 1) + 0.5 * rho_r * 0.065])
        G2l, G2r = rng.normal(size=(2, 4)) * 0.2, rng.normal(size=(2, 4)) * 0.2
        th = rng.uniform(0, 2 * np.pi)
        n2 = np.array([math.cos(th), math.sin(th)])
        delta = rng.uniform(0.05, 0.2)
        a2 = O2.gks_flux_point(spec, W2l, W2r, G2l, G2r, n2, delta)

        def lift(W):
            return np.array([W[0], W[1], W[2], 0.0, W[3]])

        def liftg(G):
            g = np.zeros((3, 5))
            for d in range(2):
                g[d] = lift(G[d])
            return g
        a3 = O3.gks_flux_point(spec, lift(W2l), lift(W2r), liftg(G2l), liftg(G2r),
                               np.array([n2[0], n2[1], 0.0]), delta)
        for x2, x3 in zip(a2, a3):
            np.testing.assert_allclose(x3[[0, 1, 2, 4]], x2, rtol=1e-11, atol=1e-13)
            assert abs(x3[3]) < 1e-13


def test_uniform_state_and_rotation_invariance(O3):
    rng = np.random.default_rng(3)
    spec = dict(gamma=GAM, mu=0.02)
    for _ in range(4):
        W = rand_state(rng)
        n = rand_normal(rng)
        z = np.zeros((3, 5))
        F0, F1, Wc, Wt = O3.gks_flux_point(spec, W, W, z, z, n)
        np.testing.assert_allclose(F0, euler3(W, n), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(F1, 0.0, atol=1e-14)
        np.testing.assert_allclose(Wt, 0.0, atol=1e-14)
        # rotate the whole problem by a random rotation Q
        Wl, Wr = rand_state(rng), rand_state(rng)
        Gl, Gr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))

        def rotW(W):
            return np.concatenate([[W[0]], Q @ W[1:4], [W[4]]])

        def rotG(G):
            # G[d][v]: derivative along x_d of W_v; rotated field W'(x) = R W(Q^T x)
            Gv = np.array([rotW(G[d]) for d in range(3)])       # rotate the vector components
            return Q @ Gv                                        # rotate the derivative direction
        a = O3.gks_flux_point(spec, Wl, Wr, Gl, Gr, n, 0.1)
        b = O3.gks_flux_point(spec, rotW(Wl), rotW(Wr), rotG(Gl), rotG(Gr), Q @ n, 0.1)
        for x, y in zip(a, b):
            np.testing.assert_allclose(y, rotW(x), rtol=1e-11, atol=1e-12)


def cjac5(W, n):
    J = np.zeros((5, 5))
    for k in range(5):
        Wc = W.astype(complex)
        Wc[k] += 1e-30j
        J[:, k] = np.imag(euler3(Wc, n)) / 1e-30
    return J


@pytest.mark.parametrize("seed", [5, 6])
def test_chapman_enskog_navier_stokes_3d(O3, seed):
    """Linear field: F0 = Euler flux - (0, sigma.n, u.sigma.n + kappa dT/dn),
    sigma = mu (grad u + grad u^T - 2/N div u I), kappa = mu (N+2)/2,
    N = K + 3; W_t = -sum_d A_d W_{x_d}; F1 = A_n W_t."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.001, 0.05)
    spec = dict(gamma=GAM, mu=mu)
    W = rand_state(rng, ma=0.5)
    G = rng.normal(size=(3, 5)) * 0.3
    n = rand_normal(rng)
    F0, F1, Wc, Wt = O3.gks_flux_point(spec, W, W, G, G, n)
    E = np.eye(3)
    Wt_ref = -sum(cjac5(W, E[d]) @ G[d] for d in range(3))
    np.testing.assert_allclose(Wc, W, rtol=1e-14)
    np.testing.assert_allclose(Wt, Wt_ref, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(F1, cjac5(W, n) @ Wt_ref, rtol=1e-11, atol=1e-12)
    rho = W[0]
    u = W[1:4] / rho
    p = (GAM - 1) * (W[4] - 0.5 * rho * u @ u)
    du = np.zeros((3, 3))
    dT = np.zeros(3)
    for d in range(3):
        dr = G[d][0]
        dud = (G[d][1:4] - u * dr) / rho
        du[:, d] = dud
        dp = (GAM - 1) * (G[d][4] - 0.5 * (u @ u) * dr - rho * (u @ dud))
        dT[d] = (dp * rho - p * dr) / rho ** 2
    sigma = mu * (du + du.T - 2.0 / N_DOF * np.trace(du) * np.eye(3))
    kappa = mu * (N_DOF + 2) / 2
    sn = sigma @ n
    ref = euler3(W, n) - np.concatenate([[0.0], sn, [u @ sn + kappa * dT @ n]])
    np.testing.assert_allclose(F0, ref, rtol=1e-11, atol=1e-12)


def test_wall_ghosts(O3):
    """Slip wall: no mass or energy flux through the wall for the state and
    its ghost; no-slip: the interface state moves with the wall."""
    rng = np.random.default_rng(7)
    for _ in range(4):
        W = rand_state(rng)
        G = rng.normal(size=(3, 5)) * 0.2
        n = rand_normal(rng)
        uw = rng.normal(size=3) * 0.1
        uw -= (uw @ n) * n
        spec = dict(gamma=GAM, mu=0.01, bcs=[dict(kind="slip"), dict(kind="noslip", uw=tuple(uw))])
        Wg, Gg = O3.ghost(spec, 0, W, G, n)
        F0, _, Wc, _ = O3.gks_flux_point(spec, W, Wg, G, Gg, n)
        assert abs(F0[0]) < 1e-13 and abs(F0[4]) < 1e-12
        assert abs(Wc[1:4] @ n) < 1e-13
        Wg, Gg = O3.ghost(spec, 1, W, G, n)
        _, _, Wc, _ = O3.gks_flux_point(spec, W, Wg, G, Gg, n)
        np.testing.assert_allclose(Wc[1:4] / Wc[0], uw, atol=1e-13)


# ---------------------------------------------------------------- mesh
FT = {2: [(0, 2, 1), (0, 1, 3), (1, 2, 3), (2, 0, 3)],
      3: [(0, 2, 1), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)],
      4: [(0, 3, 2, 1), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)],
      5: [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]}

MESHES3 = {
    "tet": lambda: MG.box3(3, 3, 2, jitter=0.2, seed=1, cells="tet", tags=(0, 0, 0, 0, 0, 0)),
    "prism": lambda: MG.box3(3, 2, 3, jitter=0.2, seed=2, cells="prism", tags=(0, 0, 0, 0, 0, 0)),
    "hex": lambda: MG.box3(3, 3, 3, jitter=0.15, seed=3, cells="hex", tags=(0, 0, 0, 0, 0, 0)),
    "pyramid": lambda: MG.box3(2, 2, 2, jitter=0.15, seed=4, cells="pyramid", tags=(0, 0, 0, 0, 0, 0)),
    "sphere": lambda: MG.sphere(1, 3, 2, R_far=4.0),
}


def adjacency3(mesh):
    owners = defaultdict(list)
    for c in range(mesh.n_cells):
        nd = mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]
        for f in FT[int(mesh.cell_type[c])]:
            owners[tuple(sorted(int(nd[i]) for i in f))].append(c)
    adj = [[] for _ in range(mesh.n_cells)]
    for cs in owners.values():
        if len(cs) == 2:
            adj[cs[0]].append(cs[1]); adj[cs[1]].append(cs[0])
    return adj, owners


KEAST_A, KEAST_B = 0.5854101966249685, 0.1381966011250105


def tet_quad(P, f):
    """Exact-for-quadratics mean of f over the tet P[0..3] (4-point rule)."""
    out = 0.0
    for k in range(4):
        bar = np.full(4, KEAST_B)
        bar[k] = KEAST_A
        out += 0.25 * f(bar @ P)
    return out


@pytest.mark.parametrize("name", list(MESHES3))
def test_mesh_faces_geometry_and_ordering(O3, name):
    mesh = MESHES3[name]()
    om = O3.OracleMesh3(mesh)
    F = om.faces()
    vol, xc, M2 = om.geometry()
    adj, owners = adjacency3(mesh)
    assert om.n_faces == len(owners)
    assert int((F["c1"] < 0).sum()) == mesh.n_bfaces
    # closed cells
    acc = np.zeros((mesh.n_cells, 3))
    np.add.at(acc, F["c0"], F["S"][:, None] * F["n"])
    inner = F["c1"] >= 0
    np.add.at(acc, F["c1"][inner], -F["S"][inner, None] * F["n"][inner])
    assert np.abs(acc).max() < 1e-13
    # outward from c0: the face centre is on the positive side of c0's centroid
    xf = (F["wg"][:, :, None] * F["xg"]).sum(1)
    assert np.all(((xf - xc[F["c0"]]) * F["n"]).sum(1) > 0)
    np.testing.assert_allclose(F["wg"].sum(1), 1.0, rtol=1e-14)
    # tets: volume, centroid and second moments by an independent rule
    for c in range(mesh.n_cells):
        if mesh.cell_type[c] != MG.TET:
            continue
        P = mesh.nodes[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]]
        V = abs(np.linalg.det(P[1:] - P[0])) / 6
        assert abs(vol[c] - V) < 1e-13 * V
        cx = [tet_quad(P, lambda x, d=d: x[d]) for d in range(3)]
        np.testing.assert_allclose(xc[c], cx, atol=1e-13)
        m2 = [tet_quad(P, lambda x, i=i, j=j: (x[i] - cx[i]) * (x[j] - cx[j]))
              for i in range(3) for j in range(i, 3)]
        np.testing.assert_allclose(M2[c], m2, atol=1e-14)
    # the sweep ordering equals a restatement from the textbook definitions
    n = mesh.n_cells
    deg = [len(a) for a in adj]
    seen = [False] * n
    order = []
    while len(order) < n:
        start = min((c for c in range(n) if not seen[c]), key=lambda c: (deg[c], c))
        seen[start] = True
        q = deque([start])
        while q:
            v = q.popleft()
            order.append(v)
            for w in sorted((w for w in adj[v] if not seen[w]), key=lambda w: (deg[w], w)):
                seen[w] = True
                q.append(w)
    rcm = order[::-1]
    colour = [-1] * n
    for v in rcm:
        used = {colour[w] for w in adj[v]}
        c = 0
        while c in used:
            c += 1
        colour[v] = c
    orcm, ocol = om.ordering()
    np.testing.assert_array_equal(orcm, rcm)
    np.testing.assert_array_equal(ocol, colour)


def test_face_quadrature_is_exact_for_quadratics(O3):
    """Triangle faces: the 3-point rule against the edge-midpoint rule;
    total domain volume; box faces are planar so quad rules are exact too."""
    mesh = MESHES3["tet"]()
    om = O3.OracleMesh3(mesh)
    F = om.faces()
    vol, _, _ = om.geometry()
    assert abs(vol.sum() - 1.0) < 1e-13

    def f(x):
        return 1.0 + x[0] - 2 * x[1] + 0.5 * x[2] + x[0] * x[1] - x[2] ** 2 + 0.3 * x[0] * x[2]
    for k in range(om.n_faces):
        if F["ng"][k] != 3:
            continue
        q = sum(F["wg"][k, i] * f(F["xg"][k, i]) for i in range(3))
        # vertices from the Gauss points: x_i = 2 g_i - (g_j + g_k) ... recover them
        G = F["xg"][k, :3]
        V = np.array([2 * G[i] - G[(i + 1) % 3] - G[(i + 2) % 3] + (G.sum(0) - G[i]) * 0 for i in range(3)])
        # the symmetric rule's points are (4 v_i + v_j + v_k) / 6: invert
        Vs = np.linalg.solve(np.array([[4, 1, 1], [1, 4, 1], [1, 1, 4]]) / 6.0, G)
        mids = [(Vs[i] + Vs[(i + 1) % 3]) / 2 for i in range(3)]
        ref = sum(f(m) for m in mids) / 3
        assert abs(q - ref) < 1e-13
        area = 0.5 * np.linalg.norm(np.cross(Vs[1] - Vs[0], Vs[2] - Vs[0]))
        assert abs(area - F["S"][k]) < 1e-14


# ---------------------------------------------------------------- scheme
def quad_field(C):
    """Five quadratics (one per variable) with coefficients C[v][10]."""
    def f(x):
        m = np.array([1.0, x[0], x[1], x[2], x[0] * x[0], x[0] * x[1], x[0] * x[2], x[1] * x[1],
                      x[1] * x[2], x[2] * x[2]])
        return C @ m

    def g(x):
        dx = np.array([0, 1, 0, 0, 2 * x[0], x[1], x[2], 0, 0, 0.0])
        dy = np.array([0, 0, 1, 0, 0, x[0], 0, 2 * x[1], x[2], 0.0])
        dz = np.array([0, 0, 0, 1, 0, 0, x[0], 0, x[1], 2 * x[2]])
        return np.stack([C @ dx, C @ dy, C @ dz])
    return f, g


def test_reconstruction_exact_for_quadratics(O3):
    mesh = MG.box3(4, 4, 3, jitter=0.2, seed=8, cells="tet", tags=(0, 0, 0, 0, 0, 0))
    om = O3.OracleMesh3(mesh)
    rng = np.random.default_rng(9)
    C = rng.normal(size=(5, 10)) * 0.3
    C[:, 0] += np.array([2.0, 0.1, 0.1, 0.1, 5.0])
    f, g = quad_field(C)
    W = np.zeros((mesh.n_cells, 5))
    Wx = np.zeros((mesh.n_cells, 3, 5))
    for c in range(mesh.n_cells):
        P = mesh.nodes[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]]
        W[c] = [tet_quad(P, lambda x, v=v: f(x)[v]) for v in range(5)]
        Wx[c] = g(P.mean(0))
    s = O3.OracleSolver3(om, dict(gamma=GAM, bcs=[dict(kind="farfield", rho=1.0, u=(0.1, 0.0, 0.0), p=1 / GAM)]))
    s.set_state(W, Wx)
    s.reconstruct()
    F = om.faces()
    adj, _ = adjacency3(mesh)
    worst = 0.0
    for k in range(om.n_faces):
        c0 = F["c0"][k]
        if len(adj[c0]) < 3:
            continue
        for q in range(F["ng"][k]):
            x = F["xg"][k, q]
            v, gr = s.recon_eval(c0, x)
            worst = max(worst, np.abs(v - f(x)).max(), np.abs(gr - g(x)).max())
    assert worst < 1e-10, worst


def freestream3(n, ma=0.3):
    return np.tile(cons3(1.0, ma * 0.8, ma * 0.5, -ma * 0.3, 1 / GAM), (n, 1))


@pytest.mark.parametrize("name", ["tet", "prism", "hex", "pyramid"])
def test_free_stream_preserved(O3, name):
    mesh = MESHES3[name]()
    om = O3.OracleMesh3(mesh)
    ma = 0.3
    W0 = freestream3(mesh.n_cells, ma)
    u = W0[0, 1:4] / W0[0, 0]
    for scheme in ("S1O2", "S2O4"):
        spec = dict(gamma=GAM, mu=0.01, time_scheme=scheme,
                    bcs=[dict(kind="farfield", rho=1.0, u=tuple(u), p=1 / GAM)])
        s = O3.OracleSolver3(om, spec)
        s.set_state(W0)
        s.explicit_steps(3)
        s.pmg_cycles(2)
        W, Wx = s.get_state()
        assert np.abs(W - W0).max() < 1e-13
        assert np.abs(Wx).max() < 1e-12


def test_conservation_on_closed_slip_box(O3):
    mesh = MG.box3(3, 3, 3, jitter=0.2, seed=12, cells="prism", tags=(0, 0, 0, 0, 0, 0))
    om = O3.OracleMesh3(mesh)
    vol, xc, _ = om.geometry()
    rng = np.random.default_rng(13)
    s = O3.OracleSolver3(om, dict(gamma=GAM, mu=0.01, bcs=[dict(kind="slip")]))
    W = np.array([cons3(1 + 0.1 * math.sin(3 * x[0]), 0.1 * x[1], -0.05, 0.02 * x[2], 1 / GAM + 0.05 * x[0])
                  for x in xc])
    s.set_state(W)
    m0 = (vol[:, None] * W).sum(0)
    s.explicit_steps(4)
    W1, _ = s.get_state()
    m1 = (vol[:, None] * W1).sum(0)
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]
    assert abs(m1[4] - m0[4]) < 1e-13 * m0[4]


# ---------------------------------------------------------------- low order
def small3(O3, mu=0.01, seed=21):
    mesh = MG.box3(2, 2, 2, jitter=0.2, seed=seed, cells="prism", tags=(0, 1, 1, 0, 1, 1))
    om = O3.OracleMesh3(mesh)
    spec = dict(gamma=GAM, mu=mu, cfl_lo=1000.0,
                bcs=[dict(kind="slip"), dict(kind="farfield", rho=1.0, u=(0.3, 0.1, -0.1), p=1 / GAM)])
    s = O3.OracleSolver3(om, spec)
    rng = np.random.default_rng(seed)
    n = mesh.n_cells
    rho = rng.uniform(0.8, 1.2, n)
    U = np.array([cons3(rho[i], *rng.uniform(-0.3, 0.3, 3), rho[i] / GAM * rng.uniform(0.9, 1.1)) for i in range(n)])
    return om, s, U


def dense3(om, U, lam, D):
    F = om.faces()
    nc = U.shape[0]
    A = np.zeros((nc, 5, nc, 5))
    for i in range(nc):
        A[i, :, i, :] = D[i] * np.eye(5)
    for f in range(om.n_faces):
        c0, c1 = F["c0"][f], F["c1"][f]
        if c1 < 0:
            continue
        n, S = F["n"][f], F["S"][f]
        A[c0, :, c1, :] += S * 0.5 * (cjac5(U[c1], n) - lam[f] * np.eye(5))
        A[c1, :, c0, :] += S * 0.5 * (cjac5(U[c0], -n) - lam[f] * np.eye(5))
    return A


def test_lambda_is_spectral_radius_3d(O3):
    om, s, U = small3(O3, mu=0.0)
    lam = s.lo_lambda(U)
    F = om.faces()
    for f in range(om.n_faces):
        if F["c1"][f] < 0:
            continue
        n = F["n"][f]
        r = max(np.abs(np.linalg.eigvals(cjac5(U[F["c0"][f]], n))).max(),
                np.abs(np.linalg.eigvals(cjac5(U[F["c1"][f]], n))).max())
        assert abs(lam[f] - r) < 1e-12 * r


def test_relaxation_is_block_gauss_seidel_and_converges_to_dense_solve(O3):
    om, s, U = small3(O3, mu=0.01)
    rng = np.random.default_rng(22)
    eps = 1e-8
    R = eps * rng.normal(size=U.shape)
    lam, D = s.lo_lambda(U), s.lo_diag(U)
    A = dense3(om, U, lam, D)
    _, colour = om.ordering()
    x = np.zeros_like(U)
    for c in range(om.n_colours):
        for i in np.nonzero(colour == c)[0]:
            r = R[i].copy()
            for j in range(U.shape[0]):
                if j != i:
                    r -= A[i, :, j, :] @ x[j]
            x[i] = np.linalg.solve(A[i, :, i, :], r)
    dU = s.lo_relax(U, R, -1)
    np.testing.assert_allclose(dU / eps, x / eps, rtol=0, atol=1e-5 * np.abs(x / eps).max())
    dU = s.lo_relax(U, R, 60)
    nc = U.shape[0]
    xs = np.linalg.solve(A.reshape(5 * nc, 5 * nc), R.reshape(-1)).reshape(nc, 5)
    np.testing.assert_allclose(dU / eps, xs / eps, rtol=0, atol=1e-5 * np.abs(xs / eps).max())


def tet_average(P, f, depth=2):
    """Mean of f over the tet P by recursive 8-way subdivision and the
    4-point rule on the children (error O((h / 2**depth)^3))."""
    if depth == 0:
        return tet_quad(P, f)
    m = {(i, j): 0.5 * (P[i] + P[j]) for i in range(4) for j in range(i + 1, 4)}
    a, b, c, d = P
    kids = [np.array(t) for t in (
        (a, m[0, 1], m[0, 2], m[0, 3]), (m[0, 1], b, m[1, 2], m[1, 3]),
        (m[0, 2], m[1, 2], c, m[2, 3]), (m[0, 3], m[1, 3], m[2, 3], d),
        (m[0, 1], m[0, 2], m[0, 3], m[1, 3]), (m[0, 1], m[0, 2], m[1, 2], m[1, 3]),
        (m[0, 2], m[0, 3], m[1, 3], m[2, 3]), (m[0, 2], m[1, 2], m[1, 3], m[2, 3]))]
    vols = [abs(np.linalg.det(k[1:] - k[0])) for k in kids]
    return sum(v * tet_average(k, f, depth - 1) for v, k in zip(vols, kids)) / sum(vols)


@pytest.mark.slow
def test_high_order_on_advected_density_wave(O3):
    """Euler solution rho = 1 + 0.1 sin(2 pi (x + y + z - |U|_1 t) / L), U, p
    constant, on jittered tet boxes of two sizes: the error in the cells
    the boundary cannot reach by time T shrinks faster than second order."""
    U = np.array([0.4, 0.3, 0.2])
    k = 2 * np.pi * np.ones(3) / 1.5
    T = 0.06

    def field(t):
        def f(x):
            rho = 1 + 0.1 * np.sin(k @ x - (k @ U) * t)
            return cons3(rho, *U, 1 / GAM)
        return f
    errs = []
    for n in (6, 12):
        mesh = MG.box3(n, n, n, jitter=0.15, seed=n, cells="tet", tags=(0, 0, 0, 0, 0, 0))
        om = O3.OracleMesh3(mesh)
        vol, xc, _ = om.geometry()
        cells = [mesh.nodes[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]] for c in range(mesh.n_cells)]
        W0 = np.array([tet_average(P, field(0.0), 1) for P in cells])
        h = 1e-6
        Wx0 = np.array([[(field(0.0)(P.mean(0) + h * e) - field(0.0)(P.mean(0) - h * e)) / (2 * h)
                         for e in np.eye(3)] for P in cells])
        s = O3.OracleSolver3(om, dict(gamma=GAM, mu=0.0, time_scheme="S2O4", cfl_hi=0.3,
                                      bcs=[dict(kind="farfield", rho=1.0, u=tuple(U), p=1 / GAM)]))
        s.set_state(W0, Wx0)
        t = 0.0
        dt = 0.3 * (1.0 / n) / 2.0
        steps = int(math.ceil(T / dt))
        for _ in range(steps):
            s.highorder_step(T / steps)
        W, _ = s.get_state()
        inner = np.all((xc > 0.3) & (xc < 0.7), axis=1)
        ref = np.array([tet_average(cells[c], field(T), 1) for c in np.nonzero(inner)[0]])
        errs.append(np.abs(W[inner, 0] - ref[:, 0]).mean())
    order = math.log(errs[0] / errs[1], 2)
    assert order > 2.4, (errs, order)


def test_lf_low_level_free_stream_conservation_and_fixed_point(O3):
    """3-D Lax-Friedrichs low level: zero residual for a free stream with
    far-field ghosts, pairwise cancellation on a closed slip box, and the
    V-cycle's fixed point unchanged (the explicit step leaves the converged
    state as it is)."""
    mesh = MG.box3(2, 2, 2, jitter=0.15, seed=31, cells="prism", tags=(0, 0, 0, 0, 0, 0))
    om = O3.OracleMesh3(mesh)
    vel = (0.3, 0.1, -0.1)
    s = O3.OracleSolver3(om, dict(gamma=GAM, flux_lo="lf", bcs=[dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)]))
    U = np.tile(cons3(1.0, *vel, 1 / GAM), (mesh.n_cells, 1))
    assert np.abs(s.lo_residual(U)).max() < 1e-14
    sb = O3.OracleSolver3(om, dict(gamma=GAM, mu=0.01, flux_lo="lf", bcs=[dict(kind="slip")]))
    rng = np.random.default_rng(32)
    n = mesh.n_cells
    U = np.array([cons3(rng.uniform(0.8, 1.2), *rng.uniform(-0.3, 0.3, 3), rng.uniform(0.6, 0.8)) for _ in range(n)])
    R = sb.lo_residual(U)
    for v in (0, 4):
        assert abs(R[:, v].sum()) < 1e-14 * np.abs(R[:, v]).sum()
    # fixed point on a small far-field box with a wall
    mesh = MG.box3(2, 2, 2, jitter=0.1, seed=33, cells="prism", tags=(1, 1, 1, 1, 0, 1))
    om = O3.OracleMesh3(mesh)
    spec = dict(gamma=GAM, mu=0.02, flux_lo="lf",
                bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.2, 0.0, 0.0), p=1 / GAM)])
    s = O3.OracleSolver3(om, spec)
    s.set_state(np.tile(cons3(1.0, 0.2, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1)))
    res = s.pmg_cycles(400)
    assert res[-1] < 1e-13, res[-5:]
    W, _ = s.get_state()
    s.highorder_step()
    assert np.abs(s.get_state()[0] - W).max() < 1e-12

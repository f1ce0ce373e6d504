"""Pins of the oracle's mesh layer (Section 2.1) and of its sweep order.

Expected values come from the raw node/cell arrays: polygon areas, edge
sharing, and an independent Python restatement of reverse Cuthill-McKee
and greedy colouring from their textbook definitions.
"""
import math
from collections import defaultdict, deque

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG


def adjacency(mesh):
    """cell -> sorted neighbour list, from shared edges of the raw arrays."""
    owners = defaultdict(list)
    for c, nodes in enumerate(mesh.cells()):
        k = len(nodes)
        for i in range(k):
            a, b = int(nodes[i]), int(nodes[(i + 1) % k])
            owners[(min(a, b), max(a, b))].append(c)
    adj = [[] for _ in range(mesh.n_cells)]
    for cs in owners.values():
        if len(cs) == 2:
            adj[cs[0]].append(cs[1])
            adj[cs[1]].append(cs[0])
    return adj, owners


def rcm_and_colours(adj):
    """Reverse Cuthill-McKee (start: lowest-index cell of minimum degree;
    neighbours by (degree, index)), then greedy smallest-free colour in
    that order."""
    n = len(adj)
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
    return np.array(rcm), np.array(colour)


MESHES = {
    "cavity8": lambda: MG.cavity(8),
    "mixed": lambda: MG.box(6, 5, 0.0, 2.0, 0.0, 1.0, jitter=0.2, seed=4, cells="mixed",
                             quad_mask=lambda i, j: (i + 2 * j) % 3 == 0),
    "cylinder": lambda: MG.cylinder(24, 3, 5),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_faces_closed_cells_and_areas(oracle_lib, name):
    O = oracle_lib
    mesh = MESHES[name]()
    om = O.OracleMesh(mesh)
    F = om.faces()
    vol, xc = om.geometry()
    # each edge appears in one cell (boundary) or two cells (interior)
    adj, owners = adjacency(mesh)
    assert om.n_faces == len(owners)
    assert int((F["c1"] < 0).sum()) == mesh.n_bfaces
    # closed cells: sum_p S_p n_p = 0
    acc = np.zeros((mesh.n_cells, 2))
    for f in range(om.n_faces):
        acc[F["c0"][f]] += F["S"][f] * F["n"][f]
        if F["c1"][f] >= 0:
            acc[F["c1"][f]] -= F["S"][f] * F["n"][f]
    assert np.abs(acc).max() < 1e-14
    # areas from the shoelace formula of the raw polygons
    for c, nodes in enumerate(mesh.cells()):
        P = mesh.nodes[nodes]
        a = 0.5 * np.sum(P[:, 0] * np.roll(P[:, 1], -1) - np.roll(P[:, 0], -1) * P[:, 1])
        assert abs(a - vol[c]) < 1e-14 * max(1.0, abs(a))
    # normals leave c0
    mid = F["xg"].mean(axis=1)
    assert np.all(np.einsum("fd,fd->f", mid - xc[F["c0"]], F["n"]) > 0)
    # boundary tags match the raw boundary list
    tagmap = {}
    for b in range(mesh.n_bfaces):
        a, c = mesh.bface_nodes[2 * b], mesh.bface_nodes[2 * b + 1]
        tagmap[(min(a, c), max(a, c))] = mesh.bface_tag[b]
    assert set(F["tag"][F["c1"] < 0]) <= set(tagmap.values())
    # Gauss points: 2-point Gauss-Legendre on each edge
    for f in range(0, om.n_faces, 7):
        d = F["xg"][f, 1] - F["xg"][f, 0]
        assert abs(np.hypot(*d) - F["S"][f] / math.sqrt(3.0)) < 1e-13


def test_domain_areas(oracle_lib):
    O = oracle_lib
    vol, _ = O.OracleMesh(MG.cavity(16)).geometry()
    assert abs(vol.sum() - 1.0) < 1e-14
    n_theta = 24
    mesh = MG.cylinder(n_theta, 3, 5)
    vol, _ = O.OracleMesh(mesh).geometry()
    ring = 0.5 * n_theta * math.sin(2 * math.pi / n_theta) * (10.0 ** 2 - 0.5 ** 2)
    assert abs(vol.sum() - ring) < 1e-12 * ring


@pytest.mark.parametrize("name", list(MESHES))
def test_ordering_matches_definition(oracle_lib, name):
    O = oracle_lib
    mesh = MESHES[name]()
    om = O.OracleMesh(mesh)
    rcm, colour = om.ordering()
    adj, _ = adjacency(mesh)
    rcm_ref, col_ref = rcm_and_colours(adj)
    np.testing.assert_array_equal(rcm, rcm_ref)
    np.testing.assert_array_equal(colour, col_ref)
    # distance-1 colouring: no two neighbours share a colour
    for c in range(mesh.n_cells):
        assert all(colour[c] != colour[w] for w in adj[c])
    assert om.n_colours == colour.max() + 1


def test_configured_meshes_have_two_neighbours_everywhere():
    """The compact quadratic needs >= 2 face neighbours per cell; the
    alternating split of the cavity guarantees it at the corners."""
    for mesh in (MG.cavity(32), MG.cylinder(64, 8, 24)):
        adj, _ = adjacency(mesh)
        assert min(len(a) for a in adj) >= 2


def test_named_workload_sizes():
    assert MG.cavity(32).n_cells == 2048
    assert MG.cylinder_cells(256, 32, 96) == 57344
    r = MG.cylinder_radii()
    assert abs(r[-1] - 10.0) < 1e-12 and len(r) == 129
    t = np.diff(r)
    np.testing.assert_allclose(t[1:32] / t[:31], 1.08, rtol=1e-12)
    assert abs(t[32] / t[31] - 1.08) < 1e-12


def test_sphere_construction_of_configuration_3():
    """Icosphere level 4 (5120 triangles), 40 prism layers from 1e-3 D
    growing by 1.1, 20 split-tet layers: 512,000 cells.  With the far field
    at 5 D the outermost split prisms are about 1.5 times longer radially
    than wide (width: the mean surface triangle's edge scaled to the
    layer's mid radius); at 20 D about 3 times (the stretched outer cells
    with which the V-cycle diverges once the wake reaches them)."""
    r5 = MG.sphere_radii(40, 20, 1e-3, 1.1, 0.5, 5.0)
    r20 = MG.sphere_radii(40, 20, 1e-3, 1.1, 0.5, 20.0)
    for r, far in ((r5, 5.0), (r20, 20.0)):
        assert len(r) == 61 and abs(r[-1] - far) < 1e-12 and abs(r[0] - 0.5) < 1e-15
        t = np.diff(r)
        np.testing.assert_allclose(t[:40], 1e-3 * 1.1 ** np.arange(40), rtol=1e-12)
        assert np.all(t > 0)
    # lateral size of a level-4 surface triangle scaled to radius r: the
    # edge of the icosphere's mean triangle, sqrt(4 A / sqrt(3)), A = 4 pi R^2 / 5120
    lateral = lambda rad: math.sqrt(4.0 * (4.0 * math.pi * rad * rad / 5120) / math.sqrt(3.0))
    ratio = lambda r: np.diff(r)[-1] / lateral(0.5 * (r[-1] + r[-2]))
    assert ratio(r5) < 1.6 and ratio(r20) > 2.8
    mesh = MG.sphere(4, 40, 20, h0=1e-3, R_far=5.0)
    assert mesh.n_cells == 512000


def test_shock_reflection_case_layout():
    """Section 4's shock reflection grid: 120 x 30 quads on [0,4] x [0,1],
    tags wall (bottom), outflow (right), Dirichlet top and left; the
    initial state is the left state everywhere."""
    from paper_2109_09965_gb300 import meshgen as MG
    mesh, spec, W0 = MG.shock_reflection_case()
    assert mesh.n_cells == 3600 and mesh.n_bfaces == 300
    counts = np.bincount(mesh.bface_tag, minlength=4)
    assert list(counts) == [120, 30, 120, 30]
    kinds = [b["kind"] for b in spec["bcs"]]
    assert kinds == ["slip", "outflow", "dirichlet", "dirichlet"]
    assert spec["flux_hi"] == "full" and spec["weno_vars"] == "characteristic" and spec["mu"] == 0.0
    rho, u, v, p = MG.SR_LEFT
    np.testing.assert_allclose(W0[0], [rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * u * u])
    assert np.all(W0 == W0[0])
    assert mesh.nodes[:, 0].min() == 0.0 and mesh.nodes[:, 0].max() == 4.0 and mesh.nodes[:, 1].max() == 1.0

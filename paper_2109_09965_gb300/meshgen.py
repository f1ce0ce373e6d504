"""Seeded synthetic mesh generators (input data only).

This module produces the raw arrays a user hands to ``cgks_mesh_create``:
node coordinates, cell connectivity (VTK node order, counter-clockwise in
2-D) and tagged boundary edges.  It is the one module that both the CUDA
library's tests and the CPU oracle's tests read their inputs from, so it
deliberately contains none of the scheme's arithmetic: no face extraction,
no geometry beyond node placement, no reconstruction, no fluxes.

Meshes follow the workloads of the paper's test section (Section 4) as
re-stated for synthetic inputs:

* ``cavity``   - unit square, n x n quads each split into two triangles,
                 interior nodes jittered (seeded), lid on top.
* ``cylinder`` - hybrid O-mesh around a circular cylinder: quad layers with
                 geometric growth next to the wall, split-triangle layers
                 out to the far field.
* ``box``      - rectangle of triangles / quads / both, for tests.

Cell type codes: 0 = triangle, 1 = quadrilateral.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

TRI, QUAD = 0, 1


@dataclass
class Mesh:
    """Raw unstructured mesh arrays in the layout of ``cgks_mesh_create``."""

    dim: int
    nodes: np.ndarray          # float64 [n_nodes, dim]
    cell_type: np.ndarray      # uint8   [n_cells]
    cell_ptr: np.ndarray       # int64   [n_cells + 1]
    cell_nodes: np.ndarray     # int64   [cell_ptr[-1]]
    bface_ptr: np.ndarray      # int64   [n_bfaces + 1]
    bface_nodes: np.ndarray    # int64   [bface_ptr[-1]]
    bface_tag: np.ndarray      # int32   [n_bfaces]
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.cell_type.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_bfaces(self) -> int:
        return int(self.bface_tag.shape[0])

    def cells(self):
        """Yield the node list of every cell (slow; for tests)."""
        for c in range(self.n_cells):
            yield self.cell_nodes[self.cell_ptr[c]:self.cell_ptr[c + 1]]

    def summary(self) -> str:
        nt = int((self.cell_type == TRI).sum())
        nq = int((self.cell_type == QUAD).sum())
        return (f"{self.meta.get('name', 'mesh')}: {self.n_cells} cells "
                f"({nt} tri, {nq} quad), {self.n_nodes} nodes, "
                f"{self.n_bfaces} boundary edges")


def _finish(nodes, tris, quads, bedges, btags, meta) -> Mesh:
    tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    quads = np.asarray(quads, dtype=np.int64).reshape(-1, 4)
    nt, nq = tris.shape[0], quads.shape[0]
    cell_type = np.concatenate([np.full(nq, QUAD, np.uint8), np.full(nt, TRI, np.uint8)])
    sizes = np.concatenate([np.full(nq, 4, np.int64), np.full(nt, 3, np.int64)])
    cell_ptr = np.zeros(nq + nt + 1, np.int64)
    np.cumsum(sizes, out=cell_ptr[1:])
    cell_nodes = np.concatenate([quads.reshape(-1), tris.reshape(-1)]).astype(np.int64)
    bedges = np.asarray(bedges, dtype=np.int64).reshape(-1, 2)
    bface_ptr = np.arange(0, 2 * bedges.shape[0] + 1, 2, dtype=np.int64)
    return Mesh(2, np.ascontiguousarray(nodes, dtype=np.float64), cell_type, cell_ptr,
                cell_nodes, bface_ptr, bedges.reshape(-1).copy(),
                np.asarray(btags, dtype=np.int32), meta)


def _grid_cells(nx, ny, node_id, cells, quad_mask=None):
    """Split the (nx x ny) logical grid into cells.

    ``cells``: 'tri' (alternating diagonals: '/' where i+j is even, '\\'
    otherwise, so that every corner cell of a rectangle still touches two
    other cells), 'slash' (all '/'), 'quad', or 'mixed' (quads where
    ``quad_mask`` is true, alternating triangles elsewhere).
    Node order of every cell is counter-clockwise for a right-handed grid.
    """
    tris, quads = [], []
    for j in range(ny):
        for i in range(nx):
            a, b = node_id(i, j), node_id(i + 1, j)
            c, d = node_id(i + 1, j + 1), node_id(i, j + 1)
            use_quad = cells == "quad" or (cells == "mixed" and quad_mask is not None
                                           and quad_mask(i, j))
            if use_quad:
                quads.append((a, b, c, d))
            elif cells == "slash" or (i + j) % 2 == 0:
                tris.append((a, b, c))
                tris.append((a, c, d))
            else:
                tris.append((a, b, d))
                tris.append((b, c, d))
    return tris, quads


def box(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0, *, jitter=0.0, seed=0,
        cells="tri", tags=(0, 1, 2, 3), quad_mask=None, name="box") -> Mesh:
    """Rectangle [x0,x1]x[y0,y1] with nx*ny grid cells.

    Interior nodes move by U(-jitter*h, +jitter*h) per axis (numpy PCG64,
    ``seed``).  Boundary edges carry ``tags`` = (bottom, right, top, left).
    """
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")          # [ny+1, nx+1]
    nodes = np.stack([X.reshape(-1), Y.reshape(-1)], axis=1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
        d = rng.uniform(-1.0, 1.0, size=nodes.shape) * np.array([jitter * hx, jitter * hy])
        ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).reshape(-1)
        nodes[interior] += d[interior]

    def nid(i, j):
        return j * (nx + 1) + i

    tris, quads = _grid_cells(nx, ny, nid, cells, quad_mask)
    bedges, btags = [], []
    for i in range(nx):                       # bottom, left -> right
        bedges.append((nid(i, 0), nid(i + 1, 0))); btags.append(tags[0])
    for j in range(ny):                       # right, bottom -> top
        bedges.append((nid(nx, j), nid(nx, j + 1))); btags.append(tags[1])
    for i in range(nx):                       # top, right -> left
        bedges.append((nid(nx - i, ny), nid(nx - i - 1, ny))); btags.append(tags[2])
    for j in range(ny):                       # left, top -> bottom
        bedges.append((nid(0, ny - j), nid(0, ny - j - 1))); btags.append(tags[3])
    meta = dict(name=name, nx=nx, ny=ny, jitter=jitter, seed=seed, cells=cells,
                bbox=(x0, x1, y0, y1))
    return _finish(nodes, tris, quads, bedges, btags, meta)


# Boundary tags used by the named workloads.
CAVITY_WALL, CAVITY_LID = 0, 1
CYL_WALL, CYL_FARFIELD = 0, 1
SR_WALL, SR_OUTFLOW, SR_TOP, SR_INFLOW = 0, 1, 2, 3


def shock_reflection(nx: int = 120, ny: int = 30) -> Mesh:
    """Regular shock reflection (Section 4): the rectangle [0, 4] x [0, 1]
    on an nx x ny Cartesian grid of quads (the paper's 120 x 30 x 2 is this
    grid extruded by two layers).  Tags: 0 = reflective wall (bottom),
    1 = supersonic outflow (right), 2 = Dirichlet post-shock state (top),
    3 = Dirichlet free stream (left)."""
    return box(nx, ny, 0.0, 4.0, 0.0, 1.0, cells="quad", tags=(SR_WALL, SR_OUTFLOW, SR_TOP, SR_INFLOW),
               name="shock_reflection")


# Section 4, shock reflection: free stream on the left, the state behind
# the incident oblique shock on the top, (rho, u, v, p).
SR_LEFT = (1.0, 2.9, 0.0, 1.0 / 1.4)
SR_UP = (1.69997, 2.61934, -0.50632, 1.52819)


def shock_reflection_case(nx: int = 120, ny: int = 30, weno_eps: float = 1e-2, gamma: float = 1.4,
                          weno_vars: str = "characteristic"):
    """Mesh, problem settings (the dict both the library and the oracle
    read) and initial state (the left state everywhere) of the shock
    reflection problem: inviscid, full flux of Eq. (2nd-flux), compact
    WENO with the given epsilon on characteristic variables (as the paper
    runs it) or on the conservative ones."""
    mesh = shock_reflection(nx, ny)

    def bc(kind, st=None):
        d = dict(kind=kind)
        if st is not None:
            d.update(rho=st[0], u=(st[1], st[2]), p=st[3])
        return d

    spec = dict(gamma=gamma, mu=0.0, flux_hi="full", weno_eps=weno_eps, weno_vars=weno_vars, cfl_hi=0.4,
                bcs=[bc("slip"), bc("outflow"), bc("dirichlet", SR_UP), bc("dirichlet", SR_LEFT)])
    rho, u, v, p = SR_LEFT
    w = np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])
    return mesh, spec, np.tile(w, (mesh.n_cells, 1))


def cavity(n: int = 32, *, jitter: float = 0.1, seed: int = 1) -> Mesh:
    """Lid-driven cavity: unit square, n x n quads split into 2n^2 triangles.

    Interior nodes jittered by U(-0.1h, 0.1h) per axis.  Tags: 0 = fixed
    no-slip walls (bottom, right, left), 1 = moving lid (top).
    """
    return box(n, n, 0.0, 1.0, 0.0, 1.0, jitter=jitter, seed=seed, cells="tri",
               tags=(CAVITY_WALL, CAVITY_WALL, CAVITY_LID, CAVITY_WALL), name=f"cavity{n}")


def cylinder_radii(n_theta=256, n_quad=32, n_tri=96, growth=1.08, R=0.5, R_far=10.0,
                   h0=None):
    """Ring radii of the hybrid O-mesh.

    Quad layers start at h0 (default: a quarter of the wall's circumferential
    spacing) and grow by ``growth``; the triangle layers grow geometrically
    from 1.08x the last quad layer with the ratio chosen (bisection) so the
    outermost ring sits at ``R_far``.
    """
    if h0 is None:
        h0 = 2.0 * math.pi * R / n_theta / 4.0
    t = [h0 * growth ** k for k in range(n_quad)]
    r = [R]
    for tk in t:
        r.append(r[-1] + tk)
    if n_tri > 0:
        t0 = growth * t[-1] if t else h0
        span = R_far - r[-1]
        if span <= 0:
            raise ValueError("quad layers already reach the far field")

        def total(q):
            return t0 * n_tri if abs(q - 1.0) < 1e-14 else t0 * (q ** n_tri - 1.0) / (q - 1.0)

        lo, hi = 0.5, 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if total(mid) < span:
                lo = mid
            else:
                hi = mid
        q = 0.5 * (lo + hi)
        for k in range(n_tri):
            r.append(r[-1] + t0 * q ** k)
        r[-1] = R_far
    return np.asarray(r)


def cylinder(n_theta: int = 256, n_quad: int = 32, n_tri: int = 96, *, growth=1.08,
             R=0.5, R_far=10.0, h0=None) -> Mesh:
    """Hybrid O-mesh around a cylinder of diameter 2R centred at the origin.

    ``n_quad`` quad layers next to the wall, then ``n_tri`` layers of quads
    each split along one diagonal into two triangles.  Cells:
    n_theta*(n_quad + 2*n_tri).  Tags: 0 = cylinder wall, 1 = far field.
    """
    r = cylinder_radii(n_theta, n_quad, n_tri, growth, R, R_far, h0)
    nr = r.shape[0]
    th = 2.0 * math.pi * np.arange(n_theta) / n_theta
    nodes = np.empty((nr * n_theta, 2))
    for k in range(nr):
        nodes[k * n_theta:(k + 1) * n_theta, 0] = r[k] * np.cos(th)
        nodes[k * n_theta:(k + 1) * n_theta, 1] = r[k] * np.sin(th)

    def nid(k, j):
        return k * n_theta + (j % n_theta)

    tris, quads = [], []
    for k in range(nr - 1):
        for j in range(n_theta):
            # (radial out, then angular) keeps the counter-clockwise order
            a, b, c, d = nid(k, j), nid(k + 1, j), nid(k + 1, j + 1), nid(k, j + 1)
            if k < n_quad:
                quads.append((a, b, c, d))
            else:
                tris.append((a, b, c))
                tris.append((a, c, d))
    bedges, btags = [], []
    for j in range(n_theta):                 # wall: interior on the outside
        bedges.append((nid(0, j + 1), nid(0, j))); btags.append(CYL_WALL)
    for j in range(n_theta):
        bedges.append((nid(nr - 1, j), nid(nr - 1, j + 1))); btags.append(CYL_FARFIELD)
    meta = dict(name=f"cylinder{n_theta}x{n_quad}+{n_tri}", n_theta=n_theta,
                n_quad=n_quad, n_tri=n_tri, growth=growth, R=R, R_far=R_far)
    return _finish(nodes, tris, quads, bedges, btags, meta)


def cylinder_growth_isotropic(n_theta: int, n_quad: int, *, R: float = 0.5, cap: float = 1.08) -> float:
    """Quad-layer growth of an O-mesh family scaled by N_theta: the ratio g
    (at most ``cap``) at which the last of n_quad quad layers, starting at
    a quarter of the wall's circumferential spacing, is as thick as the
    circumferential spacing at its radius, so the quad / triangle interface
    cells are about square.  With the fixed growth of the 256-cell ring
    (1.08), rings of a few hundred cells and n_quad = N_theta / 8 push the
    quad stack out to several radii and leave the triangle layers
    shrinking outwards (cells of aspect ratio in the thousands at the far
    field); this keeps every ring's grading sane.  Bisection on g."""
    h0 = 2.0 * math.pi * R / n_theta / 4.0

    def excess(g):
        r = R + h0 * (g ** n_quad - 1.0) / (g - 1.0)
        return h0 * g ** (n_quad - 1) - 2.0 * math.pi * r / n_theta
    lo, hi = 1.0 + 1e-9, 1.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if excess(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return min(cap, 0.5 * (lo + hi))


def cylinder_potential_state(mesh: Mesh, ma: float, aoa: float = 0.0, *, gamma: float = 1.4,
                             R: float = 0.5) -> np.ndarray:
    """Initial state for a cylinder request: the incompressible potential
    flow around a circle of radius R at the cell centres (node means),
    u - i v = U (e^{-i aoa} - R^2 e^{i aoa} / z^2), with density and
    pressure from the isentropic energy balance of a free stream with
    rho = 1, c = 1: c^2 = 1 + (gamma - 1)/2 (Ma^2 - q^2), rho = c^{2/(gamma-1)},
    p = rho c^2 / gamma (c^2 floored at 0.2 where the potential flow is
    too fast).  Conservative variables [n_cells, 4].  A starting guess
    without the impulsive start of a uniform stream at a wall; the steady
    solution does not depend on it."""
    ptr = mesh.cell_ptr
    xc = np.add.reduceat(mesh.nodes[mesh.cell_nodes], ptr[:-1], axis=0) / np.diff(ptr)[:, None]
    z = xc[:, 0] + 1j * xc[:, 1]
    w = ma * (np.exp(-1j * aoa) - R * R * np.exp(1j * aoa) / (z * z))
    u, v = w.real, -w.imag
    c2 = np.maximum(1.0 + 0.5 * (gamma - 1.0) * (ma * ma - (u * u + v * v)), 0.2)
    rho = c2 ** (1.0 / (gamma - 1.0))
    p = rho * c2 / gamma
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=1)


def cylinder_cells(n_theta: int, n_quad: int, n_tri: int) -> int:
    return n_theta * (n_quad + 2 * n_tri)


# ---------------------------------------------------------------- 3-D
# Cell type codes in 3-D and node order.  Every 3-D cell is "positive": its
# first face is counter-clockwise seen from the rest of the cell.
#   tet     (2): 0 1 2 | 3
#   prism   (3): 0 1 2 | 3 4 5        node k+3 above node k
#   pyramid (4): 0 1 2 3 | 4          apex last
#   hex     (5): 0 1 2 3 | 4 5 6 7    node k+4 above node k
TET, PRISM, PYRAMID, HEX = 2, 3, 4, 5
_NV3 = {TET: 4, PRISM: 6, PYRAMID: 5, HEX: 8}


def _finish3(nodes, cells, bfaces, btags, meta) -> Mesh:
    """cells: list of (type, node tuple); bfaces: node tuples (3 or 4)."""
    cell_type = np.array([t for t, _ in cells], np.uint8)
    sizes = np.array([len(c) for _, c in cells], np.int64)
    cell_ptr = np.zeros(len(cells) + 1, np.int64)
    np.cumsum(sizes, out=cell_ptr[1:])
    cell_nodes = np.fromiter((v for _, c in cells for v in c), np.int64, count=int(cell_ptr[-1]))
    bsz = np.array([len(f) for f in bfaces], np.int64)
    bface_ptr = np.zeros(len(bfaces) + 1, np.int64)
    np.cumsum(bsz, out=bface_ptr[1:])
    bface_nodes = np.fromiter((v for f in bfaces for v in f), np.int64, count=int(bface_ptr[-1]))
    return Mesh(3, np.ascontiguousarray(nodes, np.float64), cell_type, cell_ptr, cell_nodes,
                bface_ptr, bface_nodes, np.asarray(btags, np.int32), meta)


def _orient_tet(x, t):
    """Swap two nodes of a tet if its node order is negative."""
    a, b, c, d = t
    v = np.dot(np.cross(x[b] - x[a], x[c] - x[a]), x[d] - x[a])
    return (a, c, b, d) if v < 0 else (a, b, c, d)


# the six monotone paths from corner 000 to corner 111 of a unit cube: the
# Kuhn subdivision into tets, conforming across a structured grid
_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def box3(nx: int, ny: int, nz: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0, z0=0.0, z1=1.0, *,
         jitter=0.0, seed=0, cells="tet", tags=(0, 1, 2, 3, 4, 5), hex_mask=None, name="box3") -> Mesh:
    """Box [x0,x1]x[y0,y1]x[z0,z1] with nx*ny*nz grid cells.

    ``cells``: 'tet' (6 tets per grid cell, Kuhn subdivision), 'prism' (2
    prisms per grid cell, split along the xy diagonal), 'hex', 'pyramid' (6
    pyramids per grid cell from its centre), or 'mixed' (hexes where
    ``hex_mask(i, j, k)`` is true, tets elsewhere: only on faces where both
    sides agree, so 'mixed' takes a mask constant in k and hexes only where
    the mask holds on whole columns; boundaries then match because tets and
    hexes never share a face: a hex column is surrounded by pyramid-free
    interfaces only if the mask is constant -- use it for tests of cell
    types only).  Interior nodes move by U(-jitter*h, +jitter*h) per axis.
    Boundary faces carry ``tags`` = (x0, x1, y0, y1, z0, z1).
    """
    xs, ys, zs = np.linspace(x0, x1, nx + 1), np.linspace(y0, y1, ny + 1), np.linspace(z0, z1, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)

    def nid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        h = np.array([(x1 - x0) / nx, (y1 - y0) / ny, (z1 - z0) / nz])
        d = rng.uniform(-1.0, 1.0, size=nodes.shape) * (jitter * h)
        kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)).reshape(-1)
        nodes[interior] += d[interior]
    centres = []
    cl = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                corner = {(a, b, c): nid(i + a, j + b, k + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
                h8 = (corner[0, 0, 0], corner[1, 0, 0], corner[1, 1, 0], corner[0, 1, 0],
                      corner[0, 0, 1], corner[1, 0, 1], corner[1, 1, 1], corner[0, 1, 1])
                kind = cells
                if cells == "mixed":
                    kind = "hex" if hex_mask is not None and hex_mask(i, j, k) else "tet"
                if kind == "hex":
                    cl.append((HEX, h8))
                elif kind == "prism":
                    cl.append((PRISM, (h8[0], h8[1], h8[2], h8[4], h8[5], h8[6])))
                    cl.append((PRISM, (h8[0], h8[2], h8[3], h8[4], h8[6], h8[7])))
                elif kind == "pyramid":
                    c = len(nodes) + len(centres)
                    centres.append(nodes[list(h8)].mean(axis=0))
                    for q in ((0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)):
                        # base seen from the apex (the centre) must be counter-clockwise
                        cl.append((PYRAMID, (h8[q[0]], h8[q[3]], h8[q[2]], h8[q[1]], c)))
                else:
                    for p in _KUHN:
                        v = [0, 0, 0]
                        path = [corner[tuple(v)]]
                        for ax in p:
                            v[ax] = 1
                            path.append(corner[tuple(v)])
                        cl.append((TET, tuple(path)))
    if centres:
        nodes = np.concatenate([nodes, np.array(centres)], axis=0)
    cl = [(t, _orient_tet(nodes, c)) if t == TET else (t, c) for t, c in cl]
    # boundary faces, by construction: grid quads on the six sides, split the
    # way the cells split them
    bf, bt = [], []

    def side(quad, tag, split):
        a, b, c, d = quad                      # (lo, lo) (hi, lo) (hi, hi) (lo, hi) in the side's axes
        if split == "quad":
            bf.append((a, b, c, d))
        else:                                  # diagonal from the lowest to the highest corner
            bf.append((a, b, c)); bf.append((a, c, d))
        bt.append(tag)
        if split != "quad":
            bt.append(tag)

    def kind_at(i, j, k):
        if cells == "mixed":
            return "hex" if hex_mask is not None and hex_mask(i, j, k) else "tet"
        return cells

    for k in range(nz):
        for j in range(ny):
            for (i, tag, ii) in ((0, tags[0], 0), (nx - 1, tags[1], nx)):
                kd = kind_at(i, j, k)
                side((nid(ii, j, k), nid(ii, j + 1, k), nid(ii, j + 1, k + 1), nid(ii, j, k + 1)), tag,
                     "quad" if kd in ("hex", "prism", "pyramid") else "tri")
    for k in range(nz):
        for i in range(nx):
            for (j, tag, jj) in ((0, tags[2], 0), (ny - 1, tags[3], ny)):
                kd = kind_at(i, j, k)
                side((nid(i, jj, k), nid(i + 1, jj, k), nid(i + 1, jj, k + 1), nid(i, jj, k + 1)), tag,
                     "quad" if kd in ("hex", "prism", "pyramid") else "tri")
    for j in range(ny):
        for i in range(nx):
            for (k, tag, kk) in ((0, tags[4], 0), (nz - 1, tags[5], nz)):
                kd = kind_at(i, j, k)
                side((nid(i, j, kk), nid(i + 1, j, kk), nid(i + 1, j + 1, kk), nid(i, j + 1, kk)), tag,
                     "quad" if kd in ("hex", "pyramid") else "tri")
    meta = dict(name=name, nx=nx, ny=ny, nz=nz, jitter=jitter, seed=seed, cells=cells,
                bbox=(x0, x1, y0, y1, z0, z1))
    return _finish3(nodes, cl, bf, bt, meta)


def icosphere(level: int):
    """Unit icosphere: 20 * 4**level triangles, outward counter-clockwise."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, float) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces, np.int64)
    # outward orientation
    cr = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = (cr * V[F].mean(axis=1)).sum(axis=1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def sphere_radii(n_prism, n_tet, h0, growth, R, R_far):
    """Ring radii: n_prism layers from h0 growing by ``growth``, then n_tet
    layers growing geometrically (ratio by bisection) to R_far, the first
    one 1.1x the last prism layer... written as the continuation ratio."""
    t = [h0 * growth ** k for k in range(n_prism)]
    r = [R]
    for d in t:
        r.append(r[-1] + d)
    if n_tet > 0:
        first = t[-1] * growth if t else h0
        span = R_far - r[-1]
        lo, hi = 1.0 + 1e-12, 10.0
        for _ in range(200):
            q = 0.5 * (lo + hi)
            s = first * (q ** n_tet - 1.0) / (q - 1.0)
            lo, hi = (q, hi) if s < span else (lo, q)
        q = 0.5 * (lo + hi)
        for k in range(n_tet):
            r.append(r[-1] + first * q ** k)
        r[-1] = R_far
    return np.array(r)


# The 6 ways of cutting a prism (0 1 2 | 3 4 5) into 3 tets, with the
# diagonal each one puts on the three quad faces (0 1 4 3), (1 2 5 4),
# (2 0 3 5): the diagonal named by its end that lies on the bottom triangle
# joined to the top of the other vertical edge.
def _prism_splits():
    out = []
    for k in range(3):
        a, b, c = k, (k + 1) % 3, (k + 2) % 3
        A, B, C_ = a + 3, b + 3, c + 3
        # two families per starting vertex
        out.append(((a, b, c, A), (b, c, A, B), (c, A, B, C_)))
        out.append(((a, b, c, A), (b, c, A, C_), (b, A, B, C_)))
    return out


def _tet_edges(t):
    return {(min(t[i], t[j]), max(t[i], t[j])) for i in range(4) for j in range(i + 1, 4)}


_PRISM_QUADS = ((0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))


def _split_local(p, x):
    """Cut prism p (6 global nodes) into 3 tets; each quad face takes the
    diagonal through its smallest global node index, so the cut conforms
    with the neighbours'.  Returns the tets as local indices 0..5, each
    positively ordered."""
    want = []
    for q in _PRISM_QUADS:
        g = [p[i] for i in q]
        m = int(np.argmin(g))
        want.append((min(q[m], q[(m + 2) % 4]), max(q[m], q[(m + 2) % 4])))
    for split in _prism_splits():
        edges = set().union(*(_tet_edges(t) for t in split))
        if all(w in edges for w in want):
            out = []
            for t in split:
                a, b, c, d = t
                v = np.dot(np.cross(x[p[b]] - x[p[a]], x[p[c]] - x[p[a]]), x[p[d]] - x[p[a]])
                out.append((a, c, b, d) if v < 0 else t)
            return out
    raise ValueError("no conforming prism split")


def sphere(level=4, n_prism=40, n_tet=20, *, h0=1e-3, growth=1.1, R=0.5, R_far=20.0) -> Mesh:
    """Hybrid shell around a sphere of diameter 2R at the origin: the
    icosphere of ``level`` (20*4**level triangles) extruded radially by
    ``n_prism`` prism layers (first height h0*2R, growth ``growth``), then
    ``n_tet`` layers of prisms each cut into 3 tets (conforming
    smallest-index rule), geometric out to R_far * 2R.
    Cells: 20*4**level * (n_prism + 3*n_tet).  Tags: 0 = sphere wall,
    1 = far field."""
    D = 2.0 * R
    V, F = icosphere(level)
    r = sphere_radii(n_prism, n_tet, h0 * D, growth, R, R_far * D)
    nv, nt = V.shape[0], F.shape[0]
    nodes = np.concatenate([V * rk for rk in r], axis=0)
    # prism of surface triangle (a, b, c) between rings k and k+1: the
    # surface triangle is counter-clockwise seen from outside, i.e. from
    # the outer triangle, so (a, b, c | a', b', c') is positive
    local = np.concatenate([F, F + nv], axis=1)              # [nt, 6] for k = 0
    cl = []
    prisms = np.concatenate([local + k * nv for k in range(n_prism)], axis=0) if n_prism else np.zeros((0, 6), np.int64)
    cl += [(PRISM, tuple(int(v) for v in row)) for row in prisms]
    if n_tet:
        # the cut depends only on the order of the surface indices, the same
        # in every layer; orientation is fixed on the first tet layer
        k0 = n_prism
        splits = [_split_local(tuple(int(v) for v in local[f] + k0 * nv), nodes) for f in range(nt)]
        tets = np.array([[list(t) for t in sp] for sp in splits], np.int64)   # [nt, 3, 4] local
        rows = np.take_along_axis(local[:, None, :].repeat(3, axis=1), tets, axis=2)  # [nt, 3, 4]
        for k in range(n_tet):
            g = (rows + (k0 + k) * nv).reshape(-1, 4)
            cl += [(TET, tuple(int(v) for v in row)) for row in g]
    nl = n_prism + n_tet
    bf = [tuple(int(v) for v in f) for f in F] + [tuple(int(nl * nv + v) for v in f) for f in F]
    bt = [0] * nt + [1] * nt
    meta = dict(name=f"sphere{level}", level=level, n_prism=n_prism, n_tet=n_tet, h0=h0, growth=growth,
                R=R, R_far=R_far)
    return _finish3(nodes, cl, bf, bt, meta)


SPHERE_WALL, SPHERE_FARFIELD = 0, 1


def sphere_potential_state(mesh: Mesh, ma: float, *, gamma: float = 1.4, R: float = 0.5,
                           delta: float = 0.0) -> np.ndarray:
    """Initial state for a sphere: the incompressible potential flow past a
    sphere of radius R with free stream Ma along x, at the cell centres
    (node means): u = Ma (e_x (1 + R^3 / (2 r^3)) - 3 R^3 x x_vec / (2 r^5)),
    damped towards a no-slip wall by tanh((r - R) / delta) when delta > 0;
    density and pressure from the isentropic energy balance of a free
    stream with rho = 1, c = 1 (c^2 floored at 0.2).  Conservative
    variables [n_cells, 5].  A starting guess without an impulsive start;
    the steady solution does not depend on it."""
    ptr = mesh.cell_ptr
    x = np.add.reduceat(mesh.nodes[mesh.cell_nodes], ptr[:-1], axis=0) / np.diff(ptr)[:, None]
    r = np.linalg.norm(x, axis=1)
    a = R ** 3 / (2.0 * r ** 3)
    vel = -3.0 * a[:, None] * x[:, 0:1] * x / (r * r)[:, None]
    vel[:, 0] += 1.0 + a
    vel *= ma
    if delta > 0.0:
        vel *= np.tanh(np.maximum(r - R, 0.0) / delta)[:, None]
    q2 = (vel * vel).sum(1)
    c2 = np.maximum(1.0 + 0.5 * (gamma - 1.0) * (ma * ma - q2), 0.2)
    rho = c2 ** (1.0 / (gamma - 1.0))
    p = rho * c2 / gamma
    return np.concatenate([rho[:, None], rho[:, None] * vel, (p / (gamma - 1.0) + 0.5 * rho * q2)[:, None]], axis=1)

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


def cylinder_cells(n_theta: int, n_quad: int, n_tri: int) -> int:
    return n_theta * (n_quad + 2 * n_tri)

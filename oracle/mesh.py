"""RWG edge table and cell division for the oracle (plain numpy).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
bench's CPU-baseline leg, never by the product library.

RWG functions (paper Sec. II-B, Eqs. (4)-(5), after Rao-Wilton-Glisson): one
per interior edge e = (u, v), u < v.  The plus triangle t+ is the one whose
counter-clockwise vertex order runs u -> v; on t+ f = l/(2A+) (r - p+), on t-
f = l/(2A-) (p- - r).  Edges are numbered in lexicographic (u, v) order.

Cell division (Sec. III-A, Fig. 2): every edge belongs to exactly one cell;
Gamma_m is the union of the supports of the cell's RWGs.  Two rules:
  * octant: cell = [x<0] + 2[y<0] + 4[z<0] on the edge midpoint, with a
    coordinate counted negative only below -1e-12 * (mesh extent);
  * rcb: recursive coordinate bisection of edge midpoints -- split the
    longest bounding-box axis (ties: x before y before z); the lower part gets
    floor(M/2) cells and round(n * floor(M/2) / M) edges of smallest
    coordinate (ties broken by edge index); recurse; cells numbered in order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RWGMesh:
    verts: np.ndarray        # (nv, 3)
    tris: np.ndarray         # (nt, 3)
    edges: np.ndarray        # (ne, 2) vertex ids u < v
    edge_tri: np.ndarray     # (ne, 2) [plus, minus] triangle
    edge_loc: np.ndarray     # (ne, 2) local edge index in those triangles
    edge_len: np.ndarray     # (ne,)
    tri_edge: np.ndarray     # (nt, 3) edge of local edge a (opposite vertex a)
    tri_sign: np.ndarray     # (nt, 3) +1 plus triangle, -1 minus triangle
    area: np.ndarray         # (nt,)
    normal: np.ndarray       # (nt, 3)

    @property
    def ne(self) -> int:
        return int(self.edges.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])


def build_rwg(verts: np.ndarray, tris: np.ndarray) -> RWGMesh:
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    nt = tris.shape[0]
    directed = {}
    for t in range(nt):
        for a in range(3):
            u, v = int(tris[t, (a + 1) % 3]), int(tris[t, (a + 2) % 3])
            if (u, v) in directed:
                raise ValueError("non-manifold or inconsistently oriented mesh")
            directed[(u, v)] = (t, a)
    keys = sorted({(min(u, v), max(u, v)) for (u, v) in directed})
    ne = len(keys)
    edges = np.array(keys, dtype=np.int32).reshape(ne, 2)
    edge_tri = np.zeros((ne, 2), np.int32)
    edge_loc = np.zeros((ne, 2), np.int32)
    tri_edge = np.zeros((nt, 3), np.int32)
    tri_sign = np.zeros((nt, 3), np.int32)
    for e, (u, v) in enumerate(keys):
        if (u, v) not in directed or (v, u) not in directed:
            raise ValueError("open mesh: edge with a single triangle")
        tp, ap = directed[(u, v)]
        tm, am = directed[(v, u)]
        edge_tri[e] = (tp, tm)
        edge_loc[e] = (ap, am)
        tri_edge[tp, ap] = e
        tri_sign[tp, ap] = 1
        tri_edge[tm, am] = e
        tri_sign[tm, am] = -1
    edge_len = np.linalg.norm(verts[edges[:, 1]] - verts[edges[:, 0]], axis=1)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    nl = np.linalg.norm(nrm, axis=1)
    return RWGMesh(verts, tris, edges, edge_tri, edge_loc, edge_len, tri_edge, tri_sign,
                   0.5 * nl, nrm / nl[:, None])


def edge_midpoints(m: RWGMesh) -> np.ndarray:
    return 0.5 * (m.verts[m.edges[:, 0]] + m.verts[m.edges[:, 1]])


def cells_octant(m: RWGMesh) -> np.ndarray:
    mid = edge_midpoints(m)
    ext = float(np.max(np.abs(m.verts)))
    neg = mid < -1e-12 * ext
    return (neg[:, 0].astype(np.int32) + 2 * neg[:, 1] + 4 * neg[:, 2]).astype(np.int32)


def cells_rcb(m: RWGMesh, ncell: int) -> np.ndarray:
    mid = edge_midpoints(m)
    cell = np.zeros(m.ne, np.int32)

    def rec(ids: np.ndarray, first: int, mcount: int):
        if mcount == 1:
            cell[ids] = first
            return
        pts = mid[ids]
        ext = pts.max(axis=0) - pts.min(axis=0)
        ax = int(np.argmax(ext))                       # first maximum: x < y < z
        order = np.lexsort((ids, pts[:, ax]))          # by coordinate, then edge index
        ml = mcount // 2
        nl = int(np.floor(len(ids) * ml / mcount + 0.5))
        rec(ids[order[:nl]], first, ml)
        rec(ids[order[nl:]], first + ml, mcount - ml)

    rec(np.arange(m.ne, dtype=np.int64), 0, ncell)
    return cell


def cell_lists(cell: np.ndarray, ncell: int):
    """Lambda_m: the edges of each cell in increasing edge index."""
    return [np.nonzero(cell == c)[0] for c in range(ncell)]

"""Mesh -> RWG basis (edges) and pulse basis (triangles). Test infrastructure (oracle).

Sec. II: the surface S is meshed with triangles and RWG functions f_n expand J_Delta, n x E,
n x H and n x H_eq; Sec. II-A: pulse functions h_n (one per triangle) expand rho_Delta.

Reading (the paper defers the basis to Rao-Wilton-Glisson 1982):
* one RWG function per edge shared by two triangles of a closed, consistently oriented surface;
* edge order: by object, then by the sorted vertex pair (a < b);
* T+ is the triangle whose counter-clockwise boundary (seen from outside) runs a -> b, v+ its
  vertex opposite the edge; T- likewise for b -> a;
* f_n = +l/(2A+) (r - v+) on T+ and -l/(2A-) (r - v-) on T-, so div f_n = +l/A+, -l/A-.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


class MeshError(ValueError):
    pass


@dataclass
class RWG:
    verts: np.ndarray      # [nv, 3]
    tris: np.ndarray       # [nt, 3]
    obj_t: np.ndarray      # [nt] object of triangle
    nobj: int
    # triangles
    area: np.ndarray       # [nt]
    normal: np.ndarray     # [nt, 3] unit outward
    centroid: np.ndarray   # [nt, 3]
    diam: np.ndarray       # [nt] longest edge
    # edges
    ev: np.ndarray         # [ne, 2] vertex ids a < b
    et: np.ndarray         # [ne, 2] (T+, T-)
    eopp: np.ndarray       # [ne, 2] opposite vertex ids (v+, v-)
    elen: np.ndarray       # [ne]
    obj_e: np.ndarray      # [ne]
    # per triangle: its three edges and the sign of the RWG there (+1 on T+, -1 on T-)
    t_edges: np.ndarray    # [nt, 3]
    t_esign: np.ndarray    # [nt, 3]
    t_evert: np.ndarray    # [nt, 3] vertex of the triangle opposite that edge

    @property
    def ne(self) -> int:
        return int(self.ev.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    def obj_edge_ranges(self):
        """(start, stop) of each object's contiguous edge range."""
        out = []
        for i in range(self.nobj):
            idx = np.nonzero(self.obj_e == i)[0]
            out.append((int(idx[0]), int(idx[-1]) + 1) if idx.size else (0, 0))
        return out

    def obj_tri_ranges(self):
        out = []
        for i in range(self.nobj):
            idx = np.nonzero(self.obj_t == i)[0]
            out.append((int(idx[0]), int(idx[-1]) + 1) if idx.size else (0, 0))
        return out


def build_rwg(verts, tris, obj, nobj) -> RWG:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    obj = np.asarray(obj, dtype=np.int64)
    if not np.all(np.isfinite(verts)):
        raise MeshError("non-finite vertex coordinates")
    nt = tris.shape[0]
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    dbl = np.linalg.norm(cr, axis=1)
    if np.any(dbl <= 0):
        raise MeshError("degenerate triangle")
    area = 0.5 * dbl
    normal = cr / dbl[:, None]
    centroid = (p0 + p1 + p2) / 3.0
    diam = np.max(np.stack([np.linalg.norm(p1 - p0, axis=1), np.linalg.norm(p2 - p1, axis=1),
                            np.linalg.norm(p0 - p2, axis=1)]), axis=0)

    # directed edges
    rec: dict[tuple[int, int], list] = {}
    for t in range(nt):
        for k in range(3):
            a, b = int(tris[t, k]), int(tris[t, (k + 1) % 3])
            opp = int(tris[t, (k + 2) % 3])
            key = (min(a, b), max(a, b))
            rec.setdefault(key, []).append((t, opp, +1 if a < b else -1, (k + 2) % 3))
    items = []
    for key, lst in rec.items():
        if len(lst) != 2:
            raise MeshError(f"edge {key} has {len(lst)} triangles (open or non-manifold surface)")
        (t1, o1, s1, k1), (t2, o2, s2, k2) = lst
        if s1 == s2:
            raise MeshError(f"inconsistent orientation at edge {key}")
        if s1 < 0:
            (t1, o1, s1, k1), (t2, o2, s2, k2) = (t2, o2, s2, k2), (t1, o1, s1, k1)
        if obj[t1] != obj[t2]:
            raise MeshError(f"edge {key} joins two objects")
        items.append((int(obj[t1]), key[0], key[1], t1, t2, o1, o2, k1, k2))
    items.sort()
    ne = len(items)
    if 2 * ne != 3 * nt:
        raise MeshError("2*N_E != 3*N_T")
    ev = np.array([[it[1], it[2]] for it in items], dtype=np.int64)
    et = np.array([[it[3], it[4]] for it in items], dtype=np.int64)
    eopp = np.array([[it[5], it[6]] for it in items], dtype=np.int64)
    obj_e = np.array([it[0] for it in items], dtype=np.int64)
    elen = np.linalg.norm(verts[ev[:, 1]] - verts[ev[:, 0]], axis=1)
    t_edges = np.full((nt, 3), -1, dtype=np.int64)
    t_esign = np.zeros((nt, 3), dtype=np.int64)
    t_evert = np.full((nt, 3), -1, dtype=np.int64)
    fill = np.zeros(nt, dtype=np.int64)
    for n, it in enumerate(items):
        for (t, opp, s) in ((it[3], it[5], +1), (it[4], it[6], -1)):
            j = fill[t]
            t_edges[t, j] = n
            t_esign[t, j] = s
            t_evert[t, j] = opp
            fill[t] += 1
    return RWG(verts, tris, obj, int(nobj), area, normal, centroid, diam,
               ev, et, eopp, elen, obj_e, t_edges, t_esign, t_evert)


def from_mesh(mesh) -> RWG:
    return build_rwg(mesh.verts, mesh.tris, mesh.obj, mesh.nobj)


def rwg_eval(rw: RWG, n, t, r):
    """f_n(r) for points r [..., 3] on triangle t (0 if t is not in the support of n)."""
    r = np.asarray(r, dtype=np.float64)
    if rw.et[n, 0] == t:
        return rw.elen[n] / (2 * rw.area[t]) * (r - rw.verts[rw.eopp[n, 0]])
    if rw.et[n, 1] == t:
        return -rw.elen[n] / (2 * rw.area[t]) * (r - rw.verts[rw.eopp[n, 1]])
    return np.zeros_like(r)

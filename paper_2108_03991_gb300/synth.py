"""Seeded synthetic inputs: conductor surface meshes, AIM grid boxes and random vectors.

This module produces the geometry and random numbers that both the CUDA path and the
test-side reference consume. It holds none of the boundary-element arithmetic: no basis
functions, no integrals, no Green's functions. Everything here is a plain description of
closed, outward-oriented triangle surfaces (Sec. II: "S is meshed with triangular
elements") and of the uniform auxiliary grid box (Sec. III-A item 1).

Units: every length is in micrometres. A mesh is a tuple of
  verts  float64 [nv, 3]
  tris   int32   [nt, 3]   counter-clockwise seen from outside (outward normal)
  obj    int32   [nt]      conductor index of each triangle, objects contiguous.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MU = 1e-6  # one micrometre in metres: the length unit of every mesh here


@dataclass
class Mesh:
    verts: np.ndarray
    tris: np.ndarray
    obj: np.ndarray
    nobj: int
    # per-object conductivity (S/m); relative permittivity and permeability are 1
    sigma: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])


@dataclass
class Grid:
    origin: np.ndarray  # float64 [3]
    h: np.ndarray       # float64 [3]
    n: np.ndarray       # int64 [3]  (nx, ny, nz)

    @property
    def npts(self) -> int:
        return int(np.prod(self.n))


# ----------------------------------------------------------------------------------
# primitive surfaces
# ----------------------------------------------------------------------------------
def box(lo, size, div):
    """Closed surface of the box [lo, lo+size] with div[a] equal intervals along axis a.

    Every face is cut into div[b] x div[c] quads, each split along the same diagonal into two
    triangles; all triangles are counter-clockwise seen from outside.
    """
    lo = np.asarray(lo, dtype=np.float64)
    size = np.asarray(size, dtype=np.float64)
    div = [int(d) for d in div]
    vid: dict[tuple[int, int, int], int] = {}
    verts: list[np.ndarray] = []

    def vertex(ijk):
        key = tuple(int(v) for v in ijk)
        i = vid.get(key)
        if i is None:
            i = len(verts)
            vid[key] = i
            verts.append(lo + size * np.array(key, dtype=np.float64) / np.array(div, dtype=np.float64))
        return i

    tris = []
    for a in range(3):
        for side in (0, 1):
            b, c = (a + 1) % 3, (a + 2) % 3
            if side == 0:
                b, c = c, b  # e_b x e_c = -e_a on the low face
            for u in range(div[b]):
                for v in range(div[c]):
                    def p(du, dv):
                        ijk = [0, 0, 0]
                        ijk[a] = side * div[a]
                        ijk[b] = u + du
                        ijk[c] = v + dv
                        return vertex(ijk)
                    p00, p10, p11, p01 = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                    tris.append((p00, p10, p11))
                    tris.append((p00, p11, p01))
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def voxel_surface(solid, a, lo=(0.0, 0.0, 0.0)):
    """Closed surface of a union of cubes of side a: solid[i, j, k] marks the cube
    lo + a [i, i+1] x [j, j+1] x [k, k+1]. Every face between a solid and an empty cube is one
    quad split into two triangles, counter-clockwise seen from the empty side (outward).
    Vertices are shared through their lattice coordinates. Cubes that touch along an edge only
    would make the surface non-manifold; the caller's shapes avoid them."""
    solid = np.asarray(solid, dtype=bool)
    lo = np.asarray(lo, dtype=np.float64)
    pad = np.pad(solid, 1)
    vid: dict[tuple[int, int, int], int] = {}
    verts: list[np.ndarray] = []

    def vertex(ijk):
        key = tuple(int(v) for v in ijk)
        i = vid.get(key)
        if i is None:
            i = len(verts)
            vid[key] = i
            verts.append(lo + a * np.array(key, dtype=np.float64))
        return i

    tris = []
    for ax in range(3):
        b, c = (ax + 1) % 3, (ax + 2) % 3
        for sgn in (1, -1):
            step = [0, 0, 0]
            step[ax] = sgn
            nb = np.roll(pad, -sgn, axis=ax)  # the neighbour on the +/- ax side
            for cell in np.argwhere(pad & ~nb):
                i0 = cell - 1  # back to unpadded indices
                base = i0.copy()
                if sgn > 0:
                    base[ax] += 1
                u, v = (b, c) if sgn > 0 else (c, b)  # e_u x e_v = sgn e_ax (outward)

                def p(du, dv):
                    ijk = base.copy()
                    ijk[u] += du
                    ijk[v] += dv
                    return vertex(ijk)
                p00, p10, p11, p01 = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def icosphere(radius, subdiv, center=(0.0, 0.0, 0.0)):
    """Sphere surface: an icosahedron refined subdiv times by midpoint splitting."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            k = cache.get(key)
            if k is None:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                k = len(verts) - 1
                cache[key] = k
            return k
        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    F = np.array(faces, dtype=np.int32)
    # orient outward
    cen = np.asarray(center, dtype=np.float64)
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(p1 - p0, p2 - p0), (p0 + p1 + p2) / 3.0 - cen)
    F[s < 0] = F[s < 0][:, [0, 2, 1]]
    return V, F


def merge(parts, sigmas):
    """Concatenate closed surfaces into one multi-object mesh (objects in input order)."""
    verts, tris, obj = [], [], []
    off = 0
    for i, (V, F) in enumerate(parts):
        verts.append(V)
        tris.append(F + off)
        obj.append(np.full(F.shape[0], i, dtype=np.int32))
        off += V.shape[0]
    return Mesh(np.concatenate(verts), np.concatenate(tris).astype(np.int32),
                np.concatenate(obj), len(parts), np.asarray(sigmas, dtype=np.float64))


def grid_box(mesh: Mesh, h, margin=1, frac=1.0 / 12.0) -> Grid:
    """Smallest uniform grid whose order-2 (3x3x3) stencils around any surface point fit.

    The origin sits `margin + frac` spacings below the mesh's bounding box, so that centroids of
    structured meshes (multiples of a sixth of a cell) never fall half-way between two nodes.
    """
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)).copy()
    lo = mesh.verts.min(axis=0)
    hi = mesh.verts.max(axis=0)
    origin = lo - (margin + frac) * h
    # largest anchor: floor((hi - origin)/h + 0.5); stencil reaches anchor + margin
    top = np.floor((hi - origin) / h + 0.5).astype(np.int64) + margin
    n = top + 1
    return Grid(origin, h, n)


# ----------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------
SIGMA_CU = 5.8e7
SIGMA_AU = 4.1e7


def bar_mesh(w, t, length, a, sigma=SIGMA_CU, lo=(0.0, 0.0, 0.0)) -> Mesh:
    """One rectangular bar w x t x length (um), structured squares of side a split in two."""
    div = (round(w / a), round(t / a), round(length / a))
    V, F = box(lo, (w, t, length), div)
    return merge([(V, F)], [sigma])


def square_loop(side, w, t, a, sigma=SIGMA_CU) -> Mesh:
    """A closed square loop (picture frame) of a conductor with cross-section w x t: outer side
    `side`, in the plane z in [0, t], meshed with squares of side a (a divides side, w, t).
    Its centreline is a square of side side - w."""
    n, m, h = round(side / a), round(w / a), round(t / a)
    solid = np.zeros((n, n, h), dtype=bool)
    solid[:, :, :] = True
    solid[m:n - m, m:n - m, :] = False
    V, F = voxel_surface(solid, a)
    return merge([(V, F)], [sigma])


def trace_batch(seed=0, ntrace=256, widths=(1.0, 4.0), lengths=(10.0, 200.0), gap=3.0, a=0.5,
                sigma=SIGMA_CU):
    """Independent copper interconnects in one structure (the batched workload): seeded straight
    and L-shaped traces of square cross-section w x w, w uniform in `widths` rounded to the mesh
    step a, centreline length lognormal clipped to `lengths` (rounded to a), laid side by side
    along y with `gap` um between their bounding boxes, meshed with a x a squares (voxel_surface).
    Each trace has two lumped ports, rings 1 um (or a quarter of the arm) in from its free ends.
    Returns the mesh and, per trace, [(axis, coord), (axis, coord)] of its port planes."""
    rng = np.random.default_rng(seed)
    parts, ports = [], []
    y0 = 0.0
    for _ in range(ntrace):
        w = max(a, round(rng.uniform(*widths) / a) * a)
        L = float(np.clip(np.exp(rng.uniform(np.log(lengths[0]), np.log(lengths[1]))), *lengths))
        L = max(4 * w, round(L / a) * a)
        lshape = bool(rng.integers(2))
        m, n = round(w / a), round(L / a)
        if lshape:  # arm 1 along x, arm 2 along +y from its far end, each about L / 2 long
            n1 = max(2 * m, n // 2)
            n2 = max(2 * m, n - n1)
            solid = np.zeros((n1, n2, m), dtype=bool)
            solid[:, :m, :] = True
            solid[n1 - m:, :, :] = True
        else:
            solid = np.ones((n, m, m), dtype=bool)
        lo = (0.0, y0, 0.0)
        V, F = voxel_surface(solid, a, lo)
        parts.append((V, F))
        inset1 = max(a, min(1.0, round(solid.shape[0] * a / 4 / a) * a))
        p1 = (0, inset1)
        if lshape:
            inset2 = max(a, min(1.0, round(solid.shape[1] * a / 4 / a) * a))
            p2 = (1, y0 + solid.shape[1] * a - inset2)
        else:
            p2 = (0, solid.shape[0] * a - inset1)
        ports.append([p1, p2])
        y0 += solid.shape[1] * a + gap
    return merge(parts, [sigma] * ntrace), ports


def split_ring(cx, cy, r_out=20.0, width=4.0, thick=1.0, gap=4.0, n_theta=50, n_r=2, n_z=1):
    """Closed surface of a split ring resonator: the annulus r_out - width <= r <= r_out in the
    plane z in [0, thick], centred at (cx, cy), with a gap of chord length `gap` (at the mean
    radius) centred on the +x direction. The ring's arc is cut into n_theta equal angular steps,
    its width into n_r and its thickness into n_z: top, bottom, outer and inner walls are quads
    of the swept cross-section and the two end faces quads of the cross-section itself, each
    split into two triangles, outward and counter-clockwise seen from outside
    (2 (2 n_theta n_r + 2 n_theta n_z + 2 n_r n_z) triangles: 608 for 50, 2, 1)."""
    r_in = r_out - width
    r_mid = r_out - 0.5 * width
    tg = 2.0 * math.asin(gap / (2.0 * r_mid))
    th = np.linspace(0.5 * tg, 2.0 * math.pi - 0.5 * tg, n_theta + 1)
    rr = np.linspace(r_in, r_out, n_r + 1)
    zz = np.linspace(0.0, thick, n_z + 1)
    vid: dict = {}
    verts: list = []

    def vertex(j, a, b):
        key = (j, a, b)
        i = vid.get(key)
        if i is None:
            i = len(verts)
            vid[key] = i
            verts.append((cx + rr[a] * math.cos(th[j]), cy + rr[a] * math.sin(th[j]), zz[b]))
        return i

    tris = []

    def quad(p00, p10, p11, p01, out):
        """Two triangles of the quad, ordered so that their normal points along `out`."""
        P = [np.array(verts[i]) for i in (p00, p10, p11)]
        nrm = np.cross(P[1] - P[0], P[2] - P[0])
        if np.dot(nrm, out) < 0:
            p10, p01 = p01, p10
        tris.append((p00, p10, p11))
        tris.append((p00, p11, p01))

    for j in range(n_theta):
        tm = 0.5 * (th[j] + th[j + 1])
        er = np.array([math.cos(tm), math.sin(tm), 0.0])
        for a in range(n_r):
            quad(vertex(j, a, n_z), vertex(j + 1, a, n_z), vertex(j + 1, a + 1, n_z),
                 vertex(j, a + 1, n_z), np.array([0.0, 0.0, 1.0]))
            quad(vertex(j, a, 0), vertex(j + 1, a, 0), vertex(j + 1, a + 1, 0), vertex(j, a + 1, 0),
                 np.array([0.0, 0.0, -1.0]))
        for b in range(n_z):
            quad(vertex(j, n_r, b), vertex(j + 1, n_r, b), vertex(j + 1, n_r, b + 1),
                 vertex(j, n_r, b + 1), er)
            quad(vertex(j, 0, b), vertex(j + 1, 0, b), vertex(j + 1, 0, b + 1), vertex(j, 0, b + 1),
                 -er)
    for j, sgn in ((0, -1.0), (n_theta, 1.0)):
        et = sgn * np.array([-math.sin(th[j]), math.cos(th[j]), 0.0])  # into the gap
        for a in range(n_r):
            for b in range(n_z):
                quad(vertex(j, a, b), vertex(j, a + 1, b), vertex(j, a + 1, b + 1),
                     vertex(j, a, b + 1), et)
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def srr_array(seed=2, nx=32, ny=32, pitch=50.0, jitter=0.05, sigma=SIGMA_AU, **ring) -> Mesh:
    """nx x ny gold split rings (the large metasurface workload): ring (i, j) centred at
    (pitch (i + 1/2), pitch (j + 1/2)), its in-plane sizes (outer radius 20 um, width 4 um, gap
    4 um) scaled by a seeded factor uniform in [1 - jitter, 1 + jitter]; thickness 1 um."""
    rng = np.random.default_rng(seed)
    scale = rng.uniform(1.0 - jitter, 1.0 + jitter, nx * ny)
    parts = []
    for i in range(nx):
        for j in range(ny):
            f = float(scale[i * ny + j])
            parts.append(split_ring(pitch * (i + 0.5), pitch * (j + 0.5), r_out=20.0 * f,
                                    width=4.0 * f, gap=4.0 * f, **ring))
    return merge(parts, [sigma] * len(parts))


def srr_array_config(seed=2, n=32, freq=1e12, pitch=50.0) -> tuple[Mesh, Grid, float]:
    """n x n gold split-ring array at 1 THz with its AIM grid (srr_grid)."""
    m = srr_array(seed, n, n, pitch)
    return m, srr_grid(n, pitch), freq


def srr_grid(n=32, pitch=50.0) -> Grid:
    """AIM grid of the n x n split-ring array: 16 n nodes along x and y (512 for 32 x 32), the
    array's n pitch spread over all but the two margin nodes (3.137 um spacing at 50 um pitch),
    8 nodes of 0.5 um along z around the 1 um thick layer; the origin is a twelfth of a cell off
    the symmetric position so that no source centre falls half-way between two nodes."""
    nxy = 16 * n
    hxy = pitch * n / (nxy - 2)
    h = np.array([hxy, hxy, 0.5])
    nn = np.array([nxy, nxy, 8], dtype=np.int64)
    centre = np.array([0.5 * pitch * n, 0.5 * pitch * n, 0.5])
    origin = centre - 0.5 * (nn - 1) * h + h / 12.0
    return Grid(origin, h, nn)


def copper_bar() -> tuple[Mesh, Grid, float]:
    """Copper bar 2x2x20 um, 0.5 um squares (1344 triangles, 2016 edges), 10 GHz,
    AIM grid spacing 0.5 um."""
    m = bar_mesh(2.0, 2.0, 20.0, 0.5)
    return m, grid_box(m, 0.5), 10e9


def bar_array_lengths(seed=0, count=16):
    rng = np.random.default_rng(seed)
    return np.round(rng.uniform(5.0, 40.0, count) * 2.0) / 2.0


def bar_array(seed=0, nx=4, ny=4, pitch=5.0, cross=1.0, a=0.5, sigma=SIGMA_CU) -> Mesh:
    """nx x ny copper bars, cross-section cross x cross um, pitch `pitch` um, seeded lengths
    uniform in [5, 40] um rounded to 0.5 um, 0.5 um squares."""
    Ls = bar_array_lengths(seed, nx * ny)
    parts = []
    for i in range(nx):
        for j in range(ny):
            L = float(Ls[i * ny + j])
            parts.append(box((i * pitch, j * pitch, 0.0), (cross, cross, L),
                             (round(cross / a), round(cross / a), round(L / a))))
    return merge(parts, [sigma] * len(parts))


def bar_array_config(seed=0, freq=10e9) -> tuple[Mesh, Grid, float]:
    """4x4 array of copper bars (precision-study workload); grid spacing 0.5 um."""
    m = bar_array(seed)
    return m, grid_box(m, 0.5), freq


def small_bars(nbars=2, length=3.0, a=0.5, pitch=2.5, sigma=SIGMA_CU) -> Mesh:
    """A few short 1x1 um bars in a row (test-sized multi-object mesh)."""
    parts = [box((i * pitch, 0.0, 0.0), (1.0, 1.0, length + 0.5 * i),
                 (round(1.0 / a), round(1.0 / a), round((length + 0.5 * i) / a)))
             for i in range(nbars)]
    return merge(parts, [sigma] * nbars)


def sphere_mesh(radius=1.0, subdiv=2, sigma=1e5) -> Mesh:
    V, F = icosphere(radius, subdiv)
    return merge([(V, F)], [sigma])


# ----------------------------------------------------------------------------------
# random vectors / matrices (seeded)
# ----------------------------------------------------------------------------------
def rand_cvec(n, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(dtype)


def rand_blocks(sizes, seed):
    """Random complex square blocks (list of [n_i, n_i] complex128)."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(max(n, 1))
            for n in sizes]

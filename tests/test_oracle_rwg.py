"""Pins of the mesh generator and the RWG / pulse data (Sec. II)."""
import os

import numpy as np
import pytest

from oracle import operators as op
from oracle.rwg import MeshError, build_rwg, from_mesh
from paper_2108_03991_gb300 import synth


def test_copper_bar_counts():
    m, g, f = synth.copper_bar()
    rw = from_mesh(m)
    assert rw.nt == 1344 and rw.ne == 2016
    assert list(g.n) == [7, 7, 43]
    assert m.nv - rw.ne + rw.nt == 2  # Euler characteristic of a sphere-like surface


def test_bar_array_counts():
    m = synth.bar_array(0)
    rw = from_mesh(m)
    assert rw.nt == 11888 and rw.ne == 17832 and rw.nobj == 16
    # edges are contiguous per object
    assert np.all(np.diff(rw.obj_e) >= 0)


def test_rwg_normal_continuity_and_divergence():
    rw = from_mesh(synth.small_bars(2, 1.0))
    n = np.arange(rw.ne)
    va, vb = rw.verts[rw.ev[:, 0]], rw.verts[rw.ev[:, 1]]
    mid = 0.5 * (va + vb)
    for side, sgn in ((0, 1.0), (1, -1.0)):
        t = rw.et[:, side]
        f = sgn * (rw.elen / (2 * rw.area[t]))[:, None] * (mid - rw.verts[rw.eopp[:, side]])
        # in-plane unit normal to the edge, pointing from T+ into T-
        e = (vb - va) / rw.elen[:, None]
        u = np.cross(e, rw.normal[t])
        u *= np.sign(np.einsum("ij,ij->i", u, rw.centroid[rw.et[:, 1]] - rw.centroid[rw.et[:, 0]]) *
                     (1 if side == 0 else 1))[:, None]
        # f . u = 1 on the edge from both sides (flux continuity of RWG functions)
        fu = np.einsum("ij,ij->i", f, np.cross(e, rw.normal[t]))
        assert np.allclose(np.abs(fu), 1.0, atol=1e-12)
    fd = op.fd_matrix(rw)
    j = synth.rand_cvec(rw.ne, 1)
    # closed surfaces carry no net charge: sum_t A_t (F D j)_t = 0 per object
    for (a, b) in rw.obj_tri_ranges():
        assert abs(np.sum(rw.area[a:b] * (fd @ j)[a:b])) < 1e-12 * np.linalg.norm(j)


def test_open_or_misoriented_mesh_rejected():
    V, F = synth.box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    with pytest.raises(MeshError):
        build_rwg(V, F[:-1], np.zeros(F.shape[0] - 1), 1)
    F2 = F.copy()
    F2[0] = F2[0][[0, 2, 1]]
    with pytest.raises(MeshError):
        build_rwg(V, F2, np.zeros(F.shape[0]), 1)
    V2 = V.copy()
    V2[0, 0] = np.nan
    with pytest.raises(MeshError):
        build_rwg(V2, F, np.zeros(F.shape[0]), 1)


def test_outward_orientation():
    m = synth.bar_mesh(1.0, 2.0, 3.0, 0.5)
    rw = from_mesh(m)
    c = m.verts.mean(axis=0)
    assert np.all(np.einsum("ij,ij->i", rw.normal, rw.centroid - c) > 0)
    # divergence theorem: sum A n . x = 3 V
    vol = np.sum(rw.area * np.einsum("ij,ij->i", rw.normal, rw.centroid)) / 3.0
    assert abs(vol - 6.0) < 1e-12


def test_voxel_surface_and_loop_topology():
    """The voxel-surface mesher reproduces the structured box (same vertices and triangles up to
    order) and meshes the square loop as one closed, consistently oriented surface of genus 1
    (V - E + F = 0)."""
    V, F = synth.voxel_surface(np.ones((2, 2, 4), dtype=bool), 0.5)
    Vb, Fb = synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 2.0), (2, 2, 4))
    assert V.shape == Vb.shape and F.shape == Fb.shape
    assert np.allclose(np.sort(V, axis=0), np.sort(Vb, axis=0))
    rw = from_mesh(synth.merge([(V, F)], [1.0]))
    assert rw.ne == 3 * rw.nt // 2
    loop = synth.square_loop(10.0, 2.0, 2.0, 1.0)
    rl = from_mesh(loop)
    assert loop.verts.shape[0] - rl.ne + rl.nt == 0


def test_sphere_mesh_counts_of_the_paper():
    """Sec. IV-A meshes its sphere with 1,956 triangles and 2,934 edges
    (tests/golden/sphere_mesh_counts.txt). Any closed genus-0 triangle mesh of that many
    triangles must give the same number of RWG functions: here the structured box of 1 x 9 x 48
    intervals (4 (1*9 + 9*48 + 48*1) = 1,956 triangles), with V - E + F = 2 (980 vertices)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "sphere_mesh_counts.txt")
    nt, ne = (int(v) for v in next(ln for ln in open(path) if ln.strip() and ln[0] != "#").split())
    mesh = synth.merge([synth.box((0.0, 0.0, 0.0), (0.5, 4.5, 24.0), (1, 9, 48))], [synth.SIGMA_CU])
    rw = from_mesh(mesh)
    assert rw.nt == nt and rw.ne == ne
    assert mesh.nv - rw.ne + rw.nt == 2 and mesh.nv == 980

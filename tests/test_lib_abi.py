"""The C-ABI library loads, exports every symbol include/bem_aim.h declares, its host-only
scheduler (Sec. III-C, Alg. 2) matches the oracle, its reverse Cuthill-McKee ordering is valid,
and aim_setup rejects invalid structures with the documented codes. No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import sched
from paper_2108_03991_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return api.lib()


def test_header_symbols_exported(L):
    src = open(os.path.join(ROOT, "include", "bem_aim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof", "defined"}
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(L, n), n
    assert set(api.SYMBOLS) <= names


@pytest.mark.parametrize("cut", [None, 20])
def test_part_schedule_matches_oracle(L, cut):
    rng = np.random.default_rng(3)
    small = rng.uniform(0.30, 0.43, 128)
    W = np.sort(np.concatenate([[small.sum() * 53 / 47], small]))[::-1]
    for P in (20, 40, 80, 160, 320, 640, 1000):
        Pi, cm = api.part_schedule(W, P, cut if cut else 0)
        Po, _, co = sched.part_schedule(W, P, cut)
        assert np.array_equal(Pi, Po)
        assert cm == co


def test_part_schedule_bus_matches_oracle(L):
    """The library's Part_Schedule on the identical-conductor buses of Sec. IV-B: two processes
    per conductor, as the oracle."""
    path = os.path.join(os.path.dirname(__file__), "golden", "bus_processes_per_conductor.txt")
    rows = [tuple(int(v) for v in ln.split()) for ln in open(path) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 7
    for pairs, P, ne in rows:
        nc = 2 * pairs
        W = np.full(nc, float(ne // nc) ** 2)
        Pi, cm = api.part_schedule(W, P, 20)
        assert np.all(Pi == 2) and cm == W[0] / 2


def test_part_schedule_rejects_unsorted(L):
    with pytest.raises(api.BemError):
        api.part_schedule(np.array([1.0, 2.0]), 4)


def test_last_error_empty_string(L):
    assert isinstance(L.bem_last_error(), bytes)


def _bandwidth(rp, ci, order):
    pos = np.empty(len(order), dtype=np.int64)
    pos[order] = np.arange(len(order))
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return int(np.max(np.abs(pos[rows] - pos[ci]))) if len(ci) else 0


def test_rcm_order_grid_graph(L):
    """The host ordering behind the sparse internal operator's band, on a 30 x 20 grid graph with
    shuffled labels: a permutation whose bandwidth is that of a row-by-row ordering (20, up to
    one), as SciPy's reverse Cuthill-McKee finds."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    nx, ny = 30, 20
    rng = np.random.default_rng(4)
    lab = rng.permutation(nx * ny)
    rows, cols = [], []
    for x in range(nx):
        for y in range(ny):
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < nx and 0 <= y + dy < ny:
                    rows.append(lab[x * ny + y])
                    cols.append(lab[(x + dx) * ny + y + dy])
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nx * ny, nx * ny))
    M.sort_indices()
    order = api.rcm_order(M.indptr, M.indices)
    assert np.array_equal(np.sort(order), np.arange(nx * ny))
    ref = reverse_cuthill_mckee(M, symmetric_mode=True)
    assert _bandwidth(M.indptr, M.indices, order) <= min(21, _bandwidth(M.indptr, M.indices, ref) + 2)


def test_rcm_order_ring_pattern(L):
    """On the kept pattern of one gold split ring at 1 THz (the oracle's reading: supports within
    23 skin depths) the half-bandwidth stays near SciPy's (113) and below the product kernel's
    limit of 192."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    from oracle import operators as op, sparse_internal as si
    from oracle.rwg import from_mesh
    from paper_2108_03991_gb300 import synth
    mesh, _, freq = synth.srr_array_config(2, 1)
    rw = from_mesh(mesh)
    delta = si.skin_depth(op.k0_of(freq), op.eps_rc(mesh.sigma[0], freq))
    M = sp.csr_matrix(si.pattern(rw, 0, rw.ne, delta))
    M.sort_indices()
    order = api.rcm_order(M.indptr, M.indices)
    assert np.array_equal(np.sort(order), np.arange(rw.ne))
    b = _bandwidth(M.indptr, M.indices, order)
    bref = _bandwidth(M.indptr, M.indices, reverse_cuthill_mckee(M, symmetric_mode=True))
    assert b <= 1.1 * bref + 2 and b <= 192


def test_rcm_order_rejects_bad_columns(L):
    with pytest.raises(api.BemError):
        api.rcm_order(np.array([0, 1, 2]), np.array([1, 5]))


# ---------------------------------------------------------------------------------------
# invalid structures: aim_setup rejects them in its host-side checks, before any device work,
# with the documented error codes (so these run without a GPU)
# ---------------------------------------------------------------------------------------
def _box():
    from paper_2108_03991_gb300 import synth
    m = synth.small_bars(1, 2.0)
    return m, synth.grid_box(m, 0.5)


def _setup_code(mesh, grid, freq=10e9, why=""):
    with pytest.raises(api.BemError) as ei:
        api.Context(mesh, grid, freq)
    assert why in str(ei.value)
    return ei.value.code


def _with(m, **kw):
    from dataclasses import replace
    return replace(m, **kw)


def test_setup_rejects_bad_values(L):
    m, g = _box()
    v = m.verts.copy()
    v[3, 1] = np.nan
    assert _setup_code(_with(m, verts=v), g, why="non-finite") == -1
    assert _setup_code(m, g, 0.0, why="frequency") == -1
    assert _setup_code(m, g, float("nan")) == -1
    assert _setup_code(_with(m, sigma=np.array([-1.0])), g, why="material") == -1
    t = m.tris.copy()
    t[5, 2] = m.verts.shape[0]
    assert _setup_code(_with(m, tris=t), g, why="out of range") == -1


def test_setup_rejects_bad_surfaces(L):
    m, g = _box()
    assert _setup_code(_with(m, tris=m.tris[:-1], obj=m.obj[:-1]), g, why="has 1 triangles") == -2
    t = m.tris.copy()
    t[7] = t[7][[0, 2, 1]]
    assert _setup_code(_with(m, tris=t), g, why="orientation") == -2  # one turned over
    extra = np.stack([m.tris[0], m.tris[0][[0, 2, 1]]])
    t = np.concatenate([m.tris, extra])
    assert _setup_code(_with(m, tris=t, obj=np.zeros(len(t), np.int32)), g,
                        why="has 4 triangles") == -2  # non-manifold
    v = m.verts.copy()
    a, b, _ = m.tris[3]
    v[b] = v[a]
    assert _setup_code(_with(m, verts=v), g, why="degenerate") == -2


def test_setup_rejects_bad_object_lists(L):
    m, g = _box()
    half = len(m.tris) // 2
    two = np.concatenate([np.zeros(half, np.int32), np.ones(len(m.tris) - half, np.int32)])
    # one closed surface cut into two objects: an edge joins them
    assert _setup_code(_with(m, obj=two, nobj=2, sigma=np.array([m.sigma[0]] * 2)), g,
                        why="joins two objects") == -2
    assert _setup_code(_with(m, obj=two[::-1].copy(), nobj=2,
                             sigma=np.array([m.sigma[0]] * 2)), g, why="non-decreasing") == -1


def test_setup_rejects_bad_grids(L):
    from dataclasses import replace
    m, g = _box()
    assert _setup_code(m, replace(g, origin=g.origin + 0.75), why="outside the grid") == -3
    assert _setup_code(m, replace(g, h=np.array([0.5, 0.0, 0.5])), why="axis 1") == -3
    assert _setup_code(m, replace(g, n=np.array([2, 9, 9])), why="axis 0") == -3

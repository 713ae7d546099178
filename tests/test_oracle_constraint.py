"""Pins of the constraint preconditioner's reading (oracle/constraint.py): with every pair in
the near region it is the dense SLIM system itself; its second block row (the continuity
equation, the constraint) is the system's at any near radius; and on three bars it cuts the
GMRES iterations of the plane-wave solve several-fold (the block-diagonal preconditioner, with
each object's exact dense operators, cuts them further; both are checked on one structure)."""
import numpy as np
import pytest

from oracle import aim as oaim, constraint, gmres, operators as op, precond
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


@pytest.fixture(scope="module")
def two_bars():
    mesh = synth.small_bars(2, 2.0, pitch=1.75)   # 0.75 um gaps: near pairs across the objects
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    S, LA, LP = op.dense_system(rw, freq, mesh.sigma)
    return dict(mesh=mesh, grid=grid, freq=freq, rw=rw, k0=k0, S=S, LA=LA, LP=LP)


def _precond(b, r_near):
    rw = b["rw"]
    A = oaim.Aim(rw, b["grid"].origin, b["grid"].h, b["grid"].n, b["k0"], r_near=r_near)
    return A, constraint.ConstraintPrecond(rw, b["freq"], b["S"].Zs, b["S"].Ys,
                                           constraint.near_part(b["LA"], A.near_e, rw.ne),
                                           constraint.near_part(b["LP"], A.near_t, rw.nt))


def test_all_pairs_near_is_the_dense_system(two_bars):
    S = two_bars["S"]
    A, M = _precond(two_bars, int(max(two_bars["grid"].n)))   # every anchor within reach
    assert len(A.near_e[0]) == two_bars["rw"].ne ** 2
    x = synth.rand_cvec(S.n, 5)
    y = S.matvec(x)
    assert np.linalg.norm(M.P @ x - y) <= 1e-12 * np.linalg.norm(y)
    assert np.linalg.norm(M(y) - x) <= 1e-6 * np.linalg.norm(x)


def test_constraint_row_is_exact(two_bars):
    """Row 2, F D (I - C) h + j k0 q, needs no external operator: P_c keeps it exactly (its C is
    formed as the product Y_eq Z; the system applies Z, then Y_eq)."""
    S, ne = two_bars["S"], two_bars["rw"].ne
    A, M = _precond(two_bars, 2)
    M_cross = np.sum(np.isin(A.near_e[0], np.arange(*two_bars["rw"].obj_edge_ranges()[0])) &
                     np.isin(A.near_e[1], np.arange(*two_bars["rw"].obj_edge_ranges()[1])))
    assert M_cross > 0   # the near region couples the two bars
    x = synth.rand_cvec(S.n, 6)
    y = S.matvec(x)[ne:]
    assert np.linalg.norm((M.P @ x)[ne:] - y) <= 1e-12 * np.linalg.norm(y)


def test_preconditioners_cut_iterations():
    """Plane-wave solve of three bars with 0.75 um gaps (near pairs across the objects), GMRES
    to 1e-6: the block-diagonal preconditioner (reading 7) needs at most 10 iterations and at
    least 10x fewer than none; the constraint preconditioner at least 4x fewer than none."""
    mesh = synth.small_bars(3, 3.0, pitch=1.75)
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    LA, LP = op.dense_rwg(rw, k0, "A"), op.dense_lphi(rw, k0)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0).build_near(LA, LP)
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    S = op.SlimSystem(rw, freq, Zs, Ys, A.LA, A.LPhi)
    Mb = precond.BlockDiagPrecond(rw, freq, Zs, Ys)
    Mc = constraint.ConstraintPrecond(rw, freq, Zs, Ys, constraint.near_part(LA, A.near_e, rw.ne),
                                      constraint.near_part(LP, A.near_t, rw.nt))
    b = np.concatenate([op.plane_wave_rhs(rw, k0) / op.ETA0, np.zeros(rw.nt)])
    _, it0, _ = gmres.gmres(S.matvec, b, tol=1e-6, restart=200, max_iter=3000)
    its = []
    for M in (Mb, Mc):
        x, it, _ = gmres.gmres(S.matvec, b, tol=1e-6, restart=200, max_iter=3000, precond=M)
        assert np.linalg.norm(S.matvec(x) - b) <= 1e-6 * np.linalg.norm(b)
        its.append(it)
    assert its[0] <= 10 and it0 >= 10 * its[0]
    assert its[1] * 4 <= it0

"""Pins of the block-diagonal preconditioner (reading of the paper's preconditioned solve)."""
import numpy as np

from oracle import aim as oaim, gmres, operators as op, precond
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


def test_single_object_block_is_exact_inverse():
    """With one object, blockdiag(A_ii^{-1}) is the inverse of the dense system."""
    mesh = synth.small_bars(1, 2.0)
    rw = from_mesh(mesh)
    freq = 10e9
    S, _, _ = op.dense_system(rw, freq, mesh.sigma)
    M = precond.BlockDiagPrecond(rw, freq, S.Zs, S.Ys)
    x = synth.rand_cvec(S.n, 3)
    y = S.matvec(x)
    assert np.linalg.norm(M(y) - x) <= 1e-6 * np.linalg.norm(x)


def test_block_preconditioner_cuts_iterations():
    mesh = synth.small_bars(3, 3.0)
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0).build_near()
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    S = op.SlimSystem(rw, freq, Zs, Ys, A.LA, A.LPhi)
    M = precond.BlockDiagPrecond(rw, freq, Zs, Ys)
    b = np.concatenate([op.plane_wave_rhs(rw, k0) / op.ETA0, np.zeros(rw.nt)])
    _, it0, _ = gmres.gmres(S.matvec, b, tol=1e-6, restart=200, max_iter=3000)
    x1, it1, _ = gmres.gmres(S.matvec, b, tol=1e-6, restart=200, max_iter=3000, precond=M)
    assert np.linalg.norm(S.matvec(x1) - b) <= 1e-6 * np.linalg.norm(b)
    assert it1 <= 10 and it0 >= 10 * it1

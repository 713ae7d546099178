"""Pins of the block-diagonal preconditioner (reading of the paper's preconditioned solve);
its effect on the iteration count is pinned beside the constraint preconditioner's
(tests/test_oracle_constraint.py)."""
import numpy as np

from oracle import operators as op, precond
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


def test_fp32_inverse_check_reading():
    """The check that decides whether a block's FP32-built inverse stands (the first
    iterative-refinement correction relative to X V, evaluated in FP32) against the exact
    forward error, on the two-bar fixture's blocks (cond ~ 7e6, mostly scaling): it bounds the
    forward error from above, stays below the 1e-2 rebuild threshold, while the residual
    ||A X V - V|| / ||V|| exceeds it for the FP32 inverse and for the FP64 inverse rounded to
    FP32 alike, so it could not tell them apart."""
    mesh = synth.small_bars(2, 2.0)
    rw = from_mesh(mesh)
    freq = 10e9
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    rng = np.random.default_rng(2)
    for (_, _, _, _, A) in precond.object_blocks(rw, freq, Zs, Ys):
        X = np.linalg.inv(A)
        A32 = A.astype(np.complex64)
        X32 = np.linalg.inv(A32)
        V = (rng.uniform(-1, 1, (len(A), 4)) + 1j * rng.uniform(-1, 1, (len(A), 4))).astype(np.complex64)
        W = X32 @ V
        corr = X32 @ (A32 @ W - V)  # all FP32, as the set-up computes it
        check = np.linalg.norm(corr) / np.linalg.norm(W)
        fwd = np.linalg.norm(W.astype(complex) - X @ V) / np.linalg.norm(X @ V)
        assert fwd <= check < 1e-2
        res32 = np.linalg.norm(A @ W.astype(complex) - V) / np.linalg.norm(V)
        Xr = X.astype(np.complex64).astype(complex)
        res_r = np.linalg.norm(A @ (Xr @ V) - V) / np.linalg.norm(V)
        assert res32 > 1e-2 and res_r > 1e-2

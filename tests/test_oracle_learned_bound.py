"""What any grid-space correction of the block-diagonal preconditioner can learn (the learned
correction M(r) = M_bd r + W net(P r); not in the paper), on the two-bar fixture, from the
oracle alone.

The target of the training is t = (A^-1 - M_bd) r, measured on the grid: |P (W g - t)|^2 /
|P t|^2. For Gaussian r the best predictor of P t from P r is linear, so the optimal grid
operator G* = (P W)^+ P K P^+ (K = A^-1 - M_bd) bounds every network. Keeping only G*'s
couplings within d grid cells (max-norm) shows what a network whose receptive field is d cells
can reach: the 4-layer 3^3 network sees 4 cells."""
import numpy as np
import pytest

from oracle import aim as oaim, gmres as og, operators as op, precond
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


@pytest.fixture(scope="module")
def bound():
    freq = 10e9
    mesh = synth.small_bars(2, 2.0)
    grid = synth.grid_box(mesh, 0.5)
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0).build_near()
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    S = op.SlimSystem(rw, freq, Zs, Ys, A.LA, A.LPhi)
    N, ne = S.n, rw.ne
    Ad = np.stack([S.matvec(e) for e in np.eye(N)], axis=1)
    M = precond.BlockDiagPrecond(rw, freq, Zs, Ys)
    Md = np.stack([M(e) for e in np.eye(N)], axis=1)
    K = np.linalg.inv(Ad) - Md
    ng = A.PP.shape[1]
    P = np.zeros((4 * ng, N))
    for c in range(3):
        P[c * ng:(c + 1) * ng, :ne] = A.PA[c].toarray().T
    P[3 * ng:, ne:] = A.PP.toarray().T
    W = P.T
    B = P @ W
    PK = P @ K
    G = np.linalg.pinv(B, rcond=1e-10) @ PK @ np.linalg.pinv(P, rcond=1e-10)
    n3 = grid.n
    i = np.arange(ng)
    ijk = np.stack([i % n3[0], (i // n3[0]) % n3[1], i // (n3[0] * n3[1])], axis=1)
    D = np.tile(np.max(np.abs(ijk[:, None, :] - ijk[None, :, :]), axis=2), (4, 4))

    def loss(d):
        Gd = np.where(D <= d, G, 0)
        return float(np.linalg.norm(B @ Gd @ P - PK) ** 2 / np.linalg.norm(PK) ** 2), Gd

    b = np.concatenate([op.plane_wave_rhs(rw, k0), np.zeros(rw.nt)])
    return dict(loss=loss, Ad=Ad, Md=Md, W=W, P=P, b=b)


def test_four_cells_learn_nothing(bound):
    """Within the network's 4 cells the optimal correction explains almost none of the target
    (the measured training loss stalls at 1.0), within 8 cells nearly all of it: the coupling
    between bars 5 cells apart is what the block-diagonal preconditioner misses."""
    l4, _ = bound["loss"](4)
    l8, _ = bound["loss"](8)
    assert l4 > 0.9
    assert l8 < 0.05


def test_grid_correction_does_not_help_fgmres(bound):
    """Even the 8-cell truncation of the optimal grid correction, added to M_bd, makes flexible
    GMRES slower than M_bd alone (4 iterations to 1e-6): the grid-projected loss is no measure of
    a preconditioner here, and M_bd leaves little to gain."""
    Ad, Md, W, P, b = bound["Ad"], bound["Md"], bound["W"], bound["P"], bound["b"]
    _, it0, _ = og.gmres(lambda x: Ad @ x, b, tol=1e-6, restart=50, max_iter=300,
                         precond=lambda r: Md @ r)
    _, G8 = bound["loss"](8)
    _, it8, _ = og.gmres(lambda x: Ad @ x, b, tol=1e-6, restart=50, max_iter=300,
                         precond=lambda r: Md @ r + W @ (G8 @ (P @ r)))
    assert it0 <= 6 and it8 > it0

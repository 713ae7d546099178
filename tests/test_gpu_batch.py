"""GPU parity on a small instance of the batched workload: independent straight and L-shaped
copper traces with two lumped ports each in one structure, 10 GHz (seed 3: three traces of
1-1.5 um cross-section and 4-8 um length, 906 RWG + 604 pulse unknowns, internal blocks of
ragged sizes). The full workload (256 traces, about 2 million RWG unknowns) is the same
generator with its default sizes. Checked against the FP64 oracle: the system matvec, the port
rings, and the 6 x 6 port admittance matrix from one device solve per port."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, operators as op, ports  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import check_system  # noqa: E402


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh, planes = synth.trace_batch(3, 3, widths=(1.0, 1.5), lengths=(4.0, 8.0))
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0).build_near()
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    S = op.SlimSystem(rw, freq, Zs, Ys, A.LA, A.LPhi)
    rings = [ports.ring_edges(rw, i, c, axis=ax) for i in range(mesh.nobj) for ax, c in planes[i]]
    return dict(ctx=ctx, rw=rw, S=S, planes=planes, rings=rings, mesh=mesh)


def test_batch_structure_and_rings(batch):
    ctx, mesh, planes = batch["ctx"], batch["mesh"], batch["planes"]
    assert ctx.nobj == 3 and len({int(np.sum(mesh.obj == i)) for i in range(3)}) == 3  # ragged
    k = 0
    for i in range(mesh.nobj):
        for ax, c in planes[i]:
            e, s = ctx.port_ring(i, ax, c)
            eo, so = batch["rings"][k]
            order = np.argsort(e)
            assert np.array_equal(e[order], np.sort(eo))
            assert np.array_equal(s[order], so[np.argsort(eo)])
            k += 1


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-7)])
def test_batch_system_matvec(batch, prec, tol):
    ctx, S = batch["ctx"], batch["S"]
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    x = synth.rand_cvec(ctx.n, 90)
    x0 = x.copy()
    x0[ctx.ne:] = 0  # q = 0: row 1 is j k0 L^A j + I_x e alone
    for mode in (-1, 2):
        ctx.matvec_schedule(mode)
        for v in (x, x0):
            y = ctx.matvec(torch.from_numpy(v.astype(npdt)).cuda(), prec=prec)
            check_system(y.cpu().numpy(), S.matvec(v), ctx.ne, tol)
    ctx.matvec_schedule(-1)


def test_batch_port_matrix(batch):
    """The 6 x 6 admittance matrix (siemens) of the three traces' ports: FP32-bulk solves to
    1e-6 with the block-diagonal preconditioner against the oracle's dense solves, within 1e-4
    of the largest entry; reciprocal; each trace's own 2 x 2 block dominates its coupling to the
    other traces."""
    ctx, rw, S = batch["ctx"], batch["rw"], batch["S"]
    Ad = S.dense()
    n = len(batch["rings"])
    Yo = np.zeros((n, n), complex)
    for q, (eq, sq) in enumerate(batch["rings"]):
        xq = np.linalg.solve(Ad, np.concatenate([ports.port_rhs(rw, eq, sq), np.zeros(rw.nt)]))
        for p, (ep, sp) in enumerate(batch["rings"]):
            Yo[p, q] = ports.port_current(rw, ep, sp, xq[:rw.ne])
    Yo /= op.ETA0  # oracle units: gap voltage eta0 * 1e-6 V, current in A / 1e-6
    Y, rc, iters = ctx.port_matrix(batch["rings"], tol=1e-6, restart=100, max_iter=500,
                                   prec_mode=api.BEM_C32, precond=1)
    assert rc == api.BEM_OK and len(iters) == n
    assert np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo)) < 1e-4
    assert np.max(np.abs(Y - Y.T)) <= 2e-3 * np.max(np.abs(Y))
    for t in range(3):
        own = np.abs(Y[2 * t:2 * t + 2, 2 * t:2 * t + 2]).max()
        other = np.abs(np.delete(Y[2 * t:2 * t + 2], [2 * t, 2 * t + 1], axis=1)).max()
        assert other < own

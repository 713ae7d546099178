"""GPU parity of the excitation and post-processing calls (bem_port_ring, bem_rhs_port,
bem_port_current, bem_farfield) against the FP64 oracle on a 1 x 1 x 4 um copper bar with two
delta-gap ports, 10 GHz. The oracle's port right-hand side s l V with V = 1 is the library's
for a gap voltage of eta0 * 1e-6 volts (micrometre scaling of the first block row); its port
current sum s l h is the library's current (amperes) times 1e6 (edge lengths in micrometres
there, metres here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, farfield, operators as op, ports  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402

Z_PORTS = (0.5, 3.5)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def bar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh = synth.bar_mesh(1.0, 1.0, 4.0, 0.5)
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0).build_near()
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    S = op.SlimSystem(rw, freq, Zs, Ys, A.LA, A.LPhi)
    rings = [ports.ring_edges(rw, 0, z) for z in Z_PORTS]
    return dict(ctx=ctx, rw=rw, k0=k0, S=S, rings=rings, Ad=S.dense())


def test_port_rings_match_oracle(bar):
    ctx = bar["ctx"]
    for z, (eo, so) in zip(Z_PORTS, bar["rings"]):
        e, s = ctx.port_ring(0, 2, z)
        order = np.argsort(e)
        assert np.array_equal(e[order], np.sort(eo))
        assert np.array_equal(s[order], so[np.argsort(eo)])
        assert len(e) == 8


def test_port_rhs_matches_oracle(bar):
    ctx, rw = bar["ctx"], bar["rw"]
    for eo, so in bar["rings"]:
        b = ctx.rhs_port(eo, so, v_gap=op.ETA0 * op.ELL, prec=api.BEM_C64).cpu().numpy()
        ref = np.concatenate([ports.port_rhs(rw, eo, so), np.zeros(rw.nt)])
        assert rel(b, ref) < 1e-14


def _oracle_admittance(bar):
    rw, Ad = bar["rw"], bar["Ad"]
    Y = np.zeros((2, 2), complex)
    for q, (eq, sq) in enumerate(bar["rings"]):
        x = np.linalg.solve(Ad, np.concatenate([ports.port_rhs(rw, eq, sq), np.zeros(rw.nt)]))
        for p, (ep, sp) in enumerate(bar["rings"]):
            Y[p, q] = ports.port_current(rw, ep, sp, x[:rw.ne])
    return Y


@pytest.mark.parametrize("mode,tol,rtol", [(api.BEM_C64, 1e-10, 1e-5), (api.BEM_C32, 1e-6, 1e-4)])
def test_two_port_admittance(bar, mode, tol, rtol):
    """Port currents from device solves (FGMRES with the block-diagonal preconditioner) against
    the oracle's dense solve of the same AIM system: within 1e-5 (FP64 solve to 1e-10) and 1e-4
    (FP32-bulk solve to 1e-6) of the largest entry; the device matrix is reciprocal."""
    ctx = bar["ctx"]
    Yo = _oracle_admittance(bar)
    Yd = np.zeros((2, 2), complex)
    for q, (eq, sq) in enumerate(bar["rings"]):
        b = ctx.rhs_port(eq, sq, v_gap=op.ETA0 * op.ELL, prec=api.BEM_C64)
        x, info = ctx.solve(b, tol=tol, restart=100, max_iter=500, prec_mode=mode, precond=1)
        assert info["status"] == 0
        for p, (ep, sp) in enumerate(bar["rings"]):
            Yd[p, q] = ctx.port_current(x, ep, sp, prec=api.BEM_C64) * 1e6
    err = np.max(np.abs(Yd - Yo)) / np.max(np.abs(Yo))
    assert err < rtol, err
    assert abs(Yd[0, 1] - Yd[1, 0]) <= 2e-3 * abs(Yd[0, 1])


@pytest.mark.parametrize("mode,tol,rtol", [(api.BEM_C64, 1e-10, 1e-5), (api.BEM_C32, 1e-6, 1e-4)])
def test_port_matrix_matches_oracle(bar, mode, tol, rtol):
    """bem_port_matrix (one device solve per port, currents of every port) against the oracle's
    dense solves: Y in siemens is the oracle's admittance (gap voltage eta0 * 1e-6 volts, current
    in amperes / 1e-6) divided by eta0."""
    ctx = bar["ctx"]
    Yo = _oracle_admittance(bar) / op.ETA0
    Y, rc, iters = ctx.port_matrix([(e, s) for e, s in bar["rings"]], tol=tol, restart=100,
                                   max_iter=500, prec_mode=mode, precond=1)
    assert rc == api.BEM_OK and len(iters) == 2 and min(iters) > 0
    assert np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo)) < rtol
    with pytest.raises(api.BemError):
        ctx.port_matrix([(np.array([ctx.ne], dtype=np.int32), np.array([1.0]))])


@pytest.mark.parametrize("prec,tol", [(api.BEM_C64, 1e-6), (api.BEM_C32, 1e-5)])
def test_farfield_matches_oracle(bar, prec, tol):
    """Radiation vector of J_Delta for a random x = [h; q], several directions. The FP64 bound
    is the Y_eq set-up discrepancy (j = h - Y Z h), the FP32 one the FP32 internal products."""
    ctx, S, rw, k0 = bar["ctx"], bar["S"], bar["rw"], bar["k0"]
    x = synth.rand_cvec(ctx.n, 3)
    rng = np.random.default_rng(4)
    rh = rng.standard_normal((5, 3))
    rh /= np.linalg.norm(rh, axis=1, keepdims=True)
    xd = torch.from_numpy(x.astype(np.complex64 if prec == api.BEM_C32 else np.complex128)).cuda()
    N = ctx.farfield(xd, rh, prec=prec)
    _, _, _, _, j = S.parts(x)
    ref = farfield.radiation_vector(rw, j, k0, rh)
    assert rel(N, ref) < tol


def test_port_errors(bar):
    ctx = bar["ctx"]
    with pytest.raises(api.BemError):
        ctx.rhs_port(np.array([ctx.ne], dtype=np.int32), np.array([1.0]))
    with pytest.raises(api.BemError):
        ctx.farfield(torch.zeros(ctx.n, dtype=torch.complex128, device="cuda"), [[1.0, 1.0, 0.0]])

"""GPU parity and behaviour of the learned correction (BF16 conv net on the AIM grid).

The network's arithmetic is BF16 storage with FP32 sums; the oracle is FP64 on the same
BF16-rounded weights and input, so the remaining difference is the BF16 rounding of the three
hidden activations (8-bit mantissas): tolerance 2e-2 relative (2-norm) per tensor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import convnet  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402


def bf16(a):
    """Round to the nearest BF16 (ties to even) through the float32 bit pattern."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("shape", [(7, 9, 11), (4, 16, 8)])
def test_convnet_forward_backward_vs_oracle(dev, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(1)
    ws = convnet.init_weights(3)
    wflat = convnet.flatten(ws).astype(np.float32)
    x = rng.standard_normal((8, nz, ny, nx)).astype(np.float32)
    g = rng.standard_normal((8, nz, ny, nx)).astype(np.float32)
    out, gw, gx = api.convnet_run(wflat, torch.from_numpy(x).to(dev), torch.from_numpy(g).to(dev))
    wsb = convnet.unflatten(bf16(wflat))
    acts = convnet.forward(bf16(x), wsb, store=bf16)
    gws, gxo = convnet.backward(acts, wsb, g.astype(np.float64))
    assert rel(out.cpu().numpy(), acts[-1]) < 1e-2
    assert rel(gx.cpu().numpy(), gxo) < 1e-2
    for l, gwl in enumerate(convnet.unflatten(gw)):
        assert rel(gwl, gws[l]) < 1e-2, l


@pytest.fixture(scope="module")
def small(dev):
    mesh = synth.small_bars(2, 2.0)
    grid = synth.grid_box(mesh, 0.5)
    ctx = api.Context(mesh, grid, 10e9)
    return ctx


def test_net_correction_vs_oracle(small):
    """z - M_bd r = W net(P r) against the oracle's P, W and network on the same weights."""
    from oracle import aim as oaim, operators as op
    from oracle.rwg import from_mesh
    ctx = small
    ctx.net_init(7)
    w = ctx.net_weights()
    r = synth.rand_cvec(ctx.n, 4).astype(np.complex64)
    rd = torch.from_numpy(r).cuda()
    corr_g = ctx.net_apply(rd, correction_only=True).cpu().numpy().astype(np.complex128)
    mesh = synth.small_bars(2, 2.0)
    grid = synth.grid_box(mesh, 0.5)
    rw = from_mesh(mesh)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, op.k0_of(10e9))
    ne = rw.ne
    nx, ny, nz = grid.n
    sig = np.stack([A.PA[c].T @ r[:ne] for c in range(3)] + [A.PP.T @ r[ne:]])
    rms = np.sqrt(np.sum(np.abs(sig) ** 2) / (8 * sig.shape[1]))
    xin = np.concatenate([[s.real, s.imag] for s in sig]).reshape(8, nz, ny, nx) / rms
    out = convnet.forward(bf16(xin), convnet.unflatten(bf16(w)), store=bf16)[-1] * rms
    phi = (out[0::2] + 1j * out[1::2]).reshape(4, -1)
    corr = np.concatenate([sum(A.PA[c] @ phi[c] for c in range(3)), A.PP @ phi[3]])
    assert rel(corr_g, corr) < 2e-2


def test_training_lowers_loss_and_solve_converges(small):
    """A few hundred Adam steps lower the training loss; FGMRES with the learned correction
    reaches the true FP64 residual of 1e-6 and does not take more iterations than the
    block-diagonal preconditioner alone (the gain is printed)."""
    ctx = small
    ctx.net_init(11)
    losses = ctx.net_train(steps=150, batch=4, lr=2e-3, seed=5)
    first, last = float(np.mean(losses[:10])), float(np.mean(losses[-10:]))
    assert np.all(np.isfinite(losses)) and last < 0.9 * first
    b = ctx.rhs_plane_wave(prec=api.BEM_C64)
    _, i1 = ctx.solve(b, tol=1e-6, restart=50, max_iter=200, prec_mode=api.BEM_C32, precond=1)
    _, i2 = ctx.solve(b, tol=1e-6, restart=50, max_iter=200, prec_mode=api.BEM_C32, precond=2)
    print(f"\nloss {first:.3e} -> {last:.3e}; iterations block {i1['iters']} learned {i2['iters']}")
    assert i2["status"] == api.BEM_OK and i2["resid_true"] <= 1e-6
    assert i2["iters"] <= i1["iters"] + 1

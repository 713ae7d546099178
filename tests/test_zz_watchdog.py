"""The solver's watchdog: restarted GMRES stops at max_iter or at its wall-time limit and returns
BEM_ENOCONV (1), not an error, with the iterate it reached and that iterate's true FP64
residual. Nothing on the device is made to fail: the limits are ordinary options."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2108_03991_gb300 import api, synth  # noqa: E402


@pytest.fixture(scope="module")
def bars():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh = synth.small_bars(2, 2.0)
    ctx = api.Context(mesh, synth.grid_box(mesh, 0.5), 10e9)
    return ctx, ctx.rhs_plane_wave(prec=api.BEM_C64)


def test_max_iter_returns_enoconv(bars):
    ctx, b = bars
    x, info = ctx.solve(b, tol=1e-14, restart=10, max_iter=20, prec_mode=api.BEM_C64)
    assert info["status"] == api.BEM_ENOCONV and info["iters"] == 20
    assert 0 < info["resid_true"] < 1 and bool(torch.isfinite(torch.view_as_real(x)).all())
    r = (b - ctx.matvec(x, prec=api.BEM_C64)).cpu().numpy()
    got = np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy())
    assert abs(got - info["resid_true"]) <= 1e-9 * max(got, 1e-30)


def test_time_limit_returns_enoconv(bars):
    ctx, b = bars
    x, info = ctx.solve(b, tol=1e-14, restart=10, max_iter=1000, prec_mode=api.BEM_C64,
                        time_limit_s=1e-9)
    assert info["status"] == api.BEM_ENOCONV and info["iters"] == 0
    assert abs(info["resid_true"] - 1.0) < 1e-12
    assert not bool(x.abs().gt(0).any())

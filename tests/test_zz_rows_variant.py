"""The row kernels' other forms (aim_rows_variant; written after the last device run and not
yet run there) against the default: form 1 (predicated near-region sums) gives the same bits,
up to the sign of zero; form 2 (the same, with two interpolation rows per warp) the same up to
rounding. L^A, L^Phi, both external operators, the system matvec and the batched system
matvec, in both precisions, on two bars whose near rows have 65-127 (L^A) and 48-80 (L^Phi)
entries: every lane ends in a partial group, and most rows take no full group at all."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2108_03991_gb300 import api, synth  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh = synth.small_bars(2, 2.0)
    c = api.Context(mesh, synth.grid_box(mesh, 0.5), 10e9)
    yield c
    c.rows_variant(0)


@pytest.mark.parametrize("prec", [api.BEM_C32, api.BEM_C64])
def test_row_kernel_forms_agree(ctx, prec):
    dt = np.complex64 if prec == api.BEM_C32 else np.complex128
    cases = [(api.AIM_OP_LA, ctx.ne), (api.AIM_OP_LPHI, ctx.nt), (api.AIM_OP_EXT, ctx.n),
             (api.AIM_OP_SYSTEM, ctx.n)]
    xs = {w: torch.from_numpy(synth.rand_cvec(n, 40 + w).astype(dt)).cuda() for w, n in cases}
    xb = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.n, 50 + r) for r in range(3)])
                          .astype(dt)).cuda()
    out = {}
    for v in (0, 1, 2):
        ctx.rows_variant(v)
        out[v] = [ctx.matvec(xs[w], which=w, prec=prec).cpu().numpy() for w, _ in cases]
        out[v].append(ctx.matvec_batch(xb, prec=prec).cpu().numpy())
    ctx.rows_variant(0)
    tol = 1e-6 if prec == api.BEM_C32 else 1e-14
    for a, b, c in zip(out[0], out[1], out[2]):
        assert np.all(np.isfinite(a)) and np.array_equal(a, b)
        assert np.linalg.norm(c - a) <= tol * np.linalg.norm(a)

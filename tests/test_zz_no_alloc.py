"""The allocation-free block GEMV (bem_blockdiag_gemv_noalloc) against bem_blockdiag_gemv.

Callers whose device memory belongs to another allocator, or that may not allocate once
running, use the no-alloc entry point; it must give the same products as the allocating one.
This file is collected last so that a run stopping at its first failure has run everything
else; it passes alone in a fresh process as well as after the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2108_03991_gb300 import api, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-13)])
def test_noalloc_matches_allocating_gemv_twice(dev, prec, tol):
    sizes = [1, 3, 5, 17, 64, 129, 1000, 7, 2053]
    N = sum(sizes)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    for call, seed in enumerate((11, 12)):  # two calls in a row, different data
        blocks = synth.rand_blocks(sizes, seed)
        nrhs = 1 + 2 * call
        A = torch.from_numpy(api.pack_blocks(blocks, npdt)).to(dev)
        x = torch.from_numpy(np.concatenate([synth.rand_cvec(N, 30 + seed + r) for r in range(nrhs)])
                             .astype(npdt)).to(dev)
        y_ref = torch.zeros(nrhs * N, dtype=api.cdtype(prec), device=dev)
        y_new = torch.full_like(y_ref, complex(np.nan, np.nan))
        api.blockdiag_gemv(sizes, A, x, y_ref, nrhs, prec)
        api.blockdiag_gemv_noalloc(sizes, A, x, y_new, nrhs, prec)
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_noalloc_rejects_oversize(dev):
    sizes = [16] * 32769  # one panel more than the fixed scratch holds
    A = torch.zeros(4, dtype=torch.complex64, device=dev)
    x = torch.zeros(4, dtype=torch.complex64, device=dev)
    y = torch.zeros(4, dtype=torch.complex64, device=dev)
    with pytest.raises(api.BemError) as ei:
        api.blockdiag_gemv_noalloc(sizes, A, x, y)
    assert ei.value.code == -1 and "scratch" in str(ei.value)

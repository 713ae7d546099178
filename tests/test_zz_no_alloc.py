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


def _both(dev, sizes, seed, nrhs, prec):
    """One call of each entry point on the same seeded blocks and vectors; returns both outputs."""
    N = sum(sizes)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    blocks = synth.rand_blocks(sizes, seed)
    A = torch.from_numpy(api.pack_blocks(blocks, npdt)).to(dev)
    x = torch.from_numpy(np.concatenate([synth.rand_cvec(N, 30 + seed + r) for r in range(nrhs)])
                         .astype(npdt)).to(dev)
    y_ref = torch.zeros(nrhs * N, dtype=api.cdtype(prec), device=dev)
    y_new = torch.full_like(y_ref, complex(np.nan, np.nan))
    api.blockdiag_gemv(sizes, A, x, y_ref, nrhs, prec)
    api.blockdiag_gemv_noalloc(sizes, A, x, y_new, nrhs, prec)
    torch.cuda.synchronize()
    return y_new.cpu().numpy(), y_ref.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-13)])
def test_noalloc_matches_allocating_gemv_twice(dev, prec, tol):
    """Two calls in a row with different data; the second has fewer row panels than the first,
    so it runs on a shorter work list over the one the first call left in the shared array."""
    first = [1, 3, 5, 17, 64, 129, 1000, 7, 2053]   # 209 panels
    second = [2053, 64, 7]                         # 134 panels
    for call, (sizes, seed) in enumerate(((first, 11), (second, 12))):
        a, b = _both(dev, sizes, seed, 1 + 2 * call, prec)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_noalloc_at_the_limit(dev):
    """Exactly 32768 panels of 16 rows (the array's capacity) is accepted and matches."""
    a, b = _both(dev, [16] * 32768, 13, 1, api.BEM_C32)
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_rejects_oversize(dev, nrhs):
    sizes = [16] * 32769  # one panel more than the fixed scratch holds
    A = torch.zeros(4, dtype=torch.complex64, device=dev)
    x = torch.zeros(4, dtype=torch.complex64, device=dev)
    y = torch.zeros(4, dtype=torch.complex64, device=dev)
    with pytest.raises(api.BemError) as ei:
        api.blockdiag_gemv_noalloc(sizes, A, x, y, nrhs)
    assert ei.value.code == -1 and "scratch" in str(ei.value)


def test_noalloc_refuses_graph_capture(dev):
    """A CUDA graph would replay the call's copy from the shared host array after other calls
    rewrote it, so the call refuses to run while its stream is capturing; outside a capture it
    still works."""
    sizes = [17, 5]
    A = torch.from_numpy(api.pack_blocks(synth.rand_blocks(sizes, 14), np.complex64)).to(dev)
    x = torch.from_numpy(synth.rand_cvec(22, 15).astype(np.complex64)).to(dev)
    y = torch.zeros(22, dtype=torch.complex64, device=dev)
    g = torch.cuda.CUDAGraph()
    with pytest.raises(api.BemError) as ei:
        with torch.cuda.graph(g):
            api.blockdiag_gemv_noalloc(sizes, A, x, y)
    assert ei.value.code == -1 and "captured" in str(ei.value)
    torch.cuda.synchronize()
    a, b = _both(dev, sizes, 14, 1, api.BEM_C32)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)

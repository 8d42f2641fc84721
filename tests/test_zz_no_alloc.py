"""GPU: the allocation-free sketch entry point, lra_sketch_noalloc.

It exists for callers that cannot allocate device memory while they run (a
service that reserves its memory budget at start-up, a host framework whose own
allocator owns the device memory).  It must produce what the context-based
lra_sketch produces, within the sketch tolerance of the parity tests
(1e-12 of max |Y|), on consecutive calls that share its static scratch array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def column_major_random(m, n, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return lra.column_major(torch.randn(m, n, generator=g, dtype=torch.float64).cuda())


CASES = [(lra.SPARSE_SIGN, 8, 0.0), (lra.SPARSE_SIGN, 16, 0.0), (lra.SPARSE_SIGN_IID, 0, 0.0),
         (lra.SPARSE_GAUSSIAN, 8, 0.0), (lra.BERNOULLI, 0, 0.01)]


@pytest.mark.parametrize("kind,zeta,p", CASES)
def test_noalloc_matches_context_sketch(kind, zeta, p):
    m, n, b, seed = 3001, 2000, 24, 77
    A = column_major_random(m, n, 5)
    f = lra.Farpca(m, n, eps=1e-2, b=b, P=1, kind=kind, zeta=zeta, p=p, seed=seed)
    # two calls in a row; the second spans several chunks of the scratch array for
    # the i.i.d. kinds (capacity n per column)
    for j0, nblk in [(0, 5), (3, 70)]:
        ref = f.sketch(A, j0, nblk).cpu().numpy()
        got = lra.sketch_noalloc(A, j0, nblk, b, kind, zeta=zeta, p=p, seed=seed).cpu().numpy()
        assert got.shape == ref.shape
        assert float(np.abs(got - ref).max()) <= 1e-12 * float(np.abs(ref).max())
    f.close()


def test_noalloc_rejects_what_does_not_fit():
    A = column_major_random(2, 100000, 1)
    # one block of an i.i.d. kind needs b * (4 + 12 n) bytes: 64 columns of n = 1e5 exceed 8 MiB
    with pytest.raises(lra.LraError) as e:
        lra.sketch_noalloc(A, 0, 1, 64, lra.SPARSE_SIGN_IID)
    assert e.value.status == lra.ERR_INVALID_ARG
    with pytest.raises(lra.LraError) as e:
        lra.sketch_noalloc(A, 0, 1, 2, lra.GAUSSIAN)
    assert e.value.status == lra.ERR_UNSUPPORTED


def test_noalloc_allocates_nothing():
    """The defining property: once the library's device code is loaded (first
    call), further calls of other shapes and chunk counts leave the device's free
    memory unchanged when the caller supplies Y."""
    m, n, b = 2500, 1800, 16
    A = column_major_random(m, n, 9)
    Ys = [torch.empty_strided((m, nblk * b), (1, m), dtype=torch.float64, device="cuda")
          for nblk in (1, 4, 40)]
    lra.sketch_noalloc(A, 0, 1, b, lra.SPARSE_SIGN, zeta=8, seed=3, Y=Ys[0])  # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for Y, (kind, zeta) in zip(Ys, [(lra.SPARSE_SIGN, 4), (lra.SPARSE_GAUSSIAN, 8),
                                    (lra.SPARSE_SIGN_IID, 0)]):
        nblk = Y.shape[1] // b
        lra.sketch_noalloc(A, 2, nblk, b, kind, zeta=zeta, seed=11, Y=Y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    # a Y of the wrong layout is refused by the binding before the library writes it
    with pytest.raises(ValueError):
        lra.sketch_noalloc(A, 0, 1, b, lra.SPARSE_SIGN, zeta=8, Y=torch.empty((m, b), dtype=torch.float64,
                                                                               device="cuda"))

"""GPU: the bounded device waits give up cleanly.

lra_selftest_waits runs an mbarrier wait (the form the tensor-core GEMM's roles
use) and the eigensolver's grid barrier against conditions that never come
true, each with a limit of 2^14 polls.  Both must give up, report the timeout,
and leave the device usable: a farPCA run and its SVD (which uses the same grid
barrier) afterwards end normally.  Nothing faults or hangs: every wait is a
bounded loop.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import low_rank_matrix  # noqa: E402
from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def test_waits_time_out_and_the_device_stays_usable():
    t0 = time.perf_counter()
    status, which = lra.selftest_waits()
    assert (status, which) == (lra.ERR_TIMEOUT, 3)
    assert time.perf_counter() - t0 < 10.0
    m, n = 1500, 900
    A = low_rank_matrix(m, n, "exp100", 3, rank=200)
    Ad = torch.empty_strided((m, n), (1, m), dtype=torch.float64, device="cuda")
    Ad.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    f = lra.Farpca(m, n, eps=1e-2, b=16, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=5)
    f.run(Ad)
    res = f.result()
    assert res["status"] == lra.OK and res["rank"] > 0
    sv = f.svd()
    assert sv["status"] == lra.OK
    s = sv["sigma"].cpu().numpy()
    ref = np.linalg.svd(A, compute_uv=False)[: len(s)]
    # Weyl: |sigma_i(QB) - sigma_i(A)| <= ||A - QB||_2 <= sqrt(E)
    assert np.all(np.abs(s - ref) <= 1.01 * np.sqrt(max(res["E"], 0.0)) + 1e-12)
    f.close()
    # a second self-test gives the same answer
    assert lra.selftest_waits() == (lra.ERR_TIMEOUT, 3)

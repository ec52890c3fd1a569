"""The allocation-free column-dot entry point (xamg_coldot_noalloc) against the
allocating one (xamg_coldot), through the C ABI.

It serves callers that cannot let the library call cudaMalloc: a framework that
has reserved all device memory for its own pool, or a latency-critical loop
that must not enter the allocator.  Its scratch is a fixed array inside the
library, so two calls in a row must both agree with the allocating entry point
(the second call finds the first call's partial sums still in the array).

This file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import build as build_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_mod.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


@pytest.mark.parametrize("n,m", [(1, 1), (4097, 3), (100003, 32), (2_000_003, 8)])
def test_noalloc_matches_allocating_coldot_twice(n, m):
    rng = np.random.default_rng(n + m)
    U = torch.from_numpy(rng.uniform(-1, 1, size=(n, m))).cuda()
    V = torch.from_numpy(rng.uniform(-1, 1, size=(n, m))).cuda()
    ref = torch.empty(m, dtype=torch.float64, device="cuda")
    B.coldot(U, V, ref)
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        B.coldot_noalloc(U, V, out)
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_more_columns_than_the_array_holds():
    U = torch.zeros((16, B.MAX_RHS + 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(B.MAX_RHS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.XamgError) as e:
        B.coldot_noalloc(U, U, out)
    assert e.value.code == B.ERR_INVALID_ARG

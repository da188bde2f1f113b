"""lspca_chain_noalloc: pass F from the library's fixed device scratch array.

For callers that may not allocate device memory at all (a host framework that
owns the GPU's memory through its own pool, or a loop that cannot take the
device synchronisation of cudaMalloc/cudaFree), the library offers pass F
with its scratch in a file-scope device array instead of a workspace.  This
test calls it through the C ABI twice in a row and compares both results with
the regular entry point lspca_chain (tensor-core path), within the tolerance
the pass-F parity tests use against the FP64 oracle (relative Frobenius
2e-6); the two no-allocation calls must agree exactly (the array keeps the
previous call's contents, which must not leak into the next result).

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest
import torch

from paper_1709_07175_gb300 import lspca as L
from paper_1709_07175_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_07175_gb300 import build
    build.build()
    c = L.Context(0)
    yield c
    c.close()


# FP32 and BF16 X, one and two M halves (k <= 128 and k = 256); (60000, 2048,
# 256) plans 38 chunks of 2 MiB partials, more than the array holds, so the
# chunk count is capped (7 chunks of 8,576 rows).
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("m,n,k", [(3001, 4096, 128), (20000, 1000, 64), (60000, 4096, 128),
                                   (3001, 2048, 256), (60000, 2048, 256)])
def test_noalloc_chain_matches_regular_path(ctx, dt, m, n, k):
    w = S.WORKLOADS["fp32_sparse"].scaled(m=m, n=n, k=k)
    X = S.generate(w).cuda().to(dt)
    U = ctx.sketch(X, k, L.omega("sparse", 0, 64))
    F_ref, _ = ctx.chain(X, U)
    outs = []
    for _ in range(2):
        F = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = L.lspca_chain_noalloc(X, U, k, F, st)
        assert rc == L.OK, L.lspca_strerror(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        outs.append(F)
    rel = lambda a, b: (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
    assert rel(outs[0], F_ref) < 2e-6
    assert rel(outs[1], F_ref) < 2e-6
    assert torch.equal(outs[0], outs[1])


def test_noalloc_rejects_oversized_and_bad_arguments(ctx):
    X = torch.zeros(64, 32768, dtype=torch.float32, device="cuda")
    U = torch.zeros(64, 256, dtype=torch.float32, device="cuda")
    F = torch.empty(256, 32768, dtype=torch.float64, device="cuda")
    # 256 x 32768 FP32 partials (32 MiB) exceed the 16 MiB array
    assert L.lspca_chain_noalloc(X, U, 256, F) == L.ERR_NOMEM
    X2 = torch.zeros(64, 32, dtype=torch.float32, device="cuda")
    U2 = torch.zeros(64, 6, dtype=torch.float32, device="cuda")
    F2 = torch.empty(6, 32, dtype=torch.float64, device="cuda")
    assert L.lspca_chain_noalloc(X2, U2, 6, F2) == L.ERR_INVALID  # k not a multiple of 4


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_noalloc_flags_non_finite_x(ctx, dt):
    """Status bit 1: a NaN in X is reported for FP32 and BF16 X alike."""
    X = torch.ones(4000, 512, dtype=dt, device="cuda")
    X[1234, 77] = float("nan")
    U = torch.ones(4000, 64, dtype=torch.float32, device="cuda")
    F = torch.empty(64, 512, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.lspca_chain_noalloc(X, U, 64, F, st) == L.OK
    torch.cuda.synchronize()
    assert int(st.item()) & 1

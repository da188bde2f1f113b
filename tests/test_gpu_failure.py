"""Failure detection without a GPU fault.

* A device wait that runs out: lspca_wait_probe waits, with the bounded
  mbarrier wait of the tensor-core pipelines, on a barrier nothing arrives at.
  The wait gives up after its limit, the status word reads LSPCA_ERR_TIMEOUT
  once (then clears), and a fit on the same context afterwards returns the
  same bits as one before it.
* A host wait that runs out: lspca_srv_wait with a zero timeout on a fit that
  needs several steps returns LSPCA_ERR_TIMEOUT, the request cannot be
  released yet (LSPCA_ERR_BUSY), and a later wait completes it with the same
  result as an undisturbed server.
"""
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


def _fit(ctx, X, w):
    r = ctx.fit(X, w.k, L.omega(w.omega, w.omega_seed, w.p), report=False)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("limit_ms", [1, 50])
def test_device_wait_times_out_and_context_recovers(ctx, limit_ms):
    w = S.WORKLOADS["fp32_sparse"].scaled(m=20000, n=1024, k=64)
    X = S.generate(w).cuda()
    before = _fit(ctx, X, w)
    assert L.lspca_sync_status(ctx.handle) == L.OK
    waited = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.lspca_wait_probe(ctx.handle, limit_ms * 1_000_000, waited) == L.OK
    assert L.lspca_sync_status(ctx.handle) == L.ERR_TIMEOUT
    assert L.lspca_sync_status(ctx.handle) == L.OK  # read once, then cleared
    ns = int(waited.item())
    assert limit_ms * 1_000_000 <= ns < limit_ms * 1_000_000 + 500_000_000
    after = _fit(ctx, X, w)
    assert L.lspca_sync_status(ctx.handle) == L.OK
    assert torch.equal(before.V, after.V) and torch.equal(before.sigma, after.sigma)


def test_wait_probe_rejects_limits_outside_range(ctx):
    assert L.lspca_wait_probe(ctx.handle, 10) == L.ERR_INVALID
    assert L.lspca_wait_probe(ctx.handle, 3_000_000_000) == L.ERR_INVALID


def test_server_wait_zero_timeout(ctx):
    w = S.WORKLOADS["fp32_sparse"].scaled(m=200_000, n=1024, k=64)  # four slices of 65,536 rows
    X = S.generate(w).cuda()
    om = L.omega(w.omega, w.omega_seed, w.p)
    srv = L.Server(0, 1 << 30, 8)
    req, V, sig = srv.submit_fit(X, w.k, om)
    assert L.lspca_srv_wait(srv.handle, req, 0) == L.ERR_TIMEOUT
    assert L.lspca_srv_release(srv.handle, req) == L.ERR_BUSY
    assert L.lspca_srv_wait(srv.handle, req, 60000) == L.OK
    torch.cuda.synchronize()
    ref_srv = L.Server(0, 1 << 30, 8)
    req2, V2, sig2 = ref_srv.submit_fit(X, w.k, om)
    assert L.lspca_srv_wait(ref_srv.handle, req2, 60000) == L.OK
    torch.cuda.synchronize()
    assert torch.equal(V, V2) and torch.equal(sig, sig2)
    assert L.lspca_srv_release(srv.handle, req) == L.OK
    srv.close()
    ref_srv.close()

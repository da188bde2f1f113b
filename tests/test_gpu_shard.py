"""Virtual row shards on one GPU (Algorithm 4's sum over row slices, the
reduction point of a multi-device fit), through the C ABI.

* S row ranges, partials summed in a fixed order, match the oracle's F and the
  unsharded fit's subspace and singular values;
* two runs give the same bits.
"""
import numpy as np
import pytest
import torch

from oracle import lspca as O
from oracle import metrics as M
from oracle import philox as P
from paper_1709_07175_gb300 import lspca as L
from paper_1709_07175_gb300 import shard
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


@pytest.mark.parametrize("wname,m,n,k,shards,tol", [("fp64_small", 2000, 500, 20, 3, 1e-12),
                                                    ("fp32_sparse", 20000, 1024, 64, 4, 1e-5)])
def test_virtual_shards_match_oracle_and_unsharded(ctx, wname, m, n, k, shards, tol):
    w = S.WORKLOADS[wname].scaled(m=m, n=n, k=k)
    X = S.generate(w).cuda()
    om = L.omega(w.omega, w.omega_seed, w.p)
    vt = torch.float64 if X.dtype == torch.float64 else torch.float32
    V, sig, rank, F, _ = shard.sharded_fit(ctx, X, m, k, om, virtual_shards=shards, vt=vt)
    V2, sig2, _, F2, _ = shard.sharded_fit(ctx, X, m, k, om, virtual_shards=shards, vt=vt)
    torch.cuda.synchronize()
    assert torch.equal(F, F2) and torch.equal(V, V2) and torch.equal(sig, sig2)

    Xd = X.double().cpu().numpy()
    Om = ctx.omega(om, n, k).cpu().numpy()  # the exact Omega bits the library used
    Fref = O.chain(O.sketch(Xd, Om), Xd)
    Fd = F.cpu().numpy()
    assert np.linalg.norm(Fd - Fref) <= tol * np.linalg.norm(Fref)

    full = ctx.fit(X, k, om, report=False)
    torch.cuda.synchronize()
    assert int(rank.item()) == int(full.rank.item())
    assert M.max_sine(full.V.double().cpu().numpy(), V.double().cpu().numpy()) < 10 * tol
    s1, s2 = sig.cpu().numpy(), full.sigma.cpu().numpy()
    assert np.max(np.abs(s1 - s2) / s2) < tol


@pytest.mark.parametrize("nparts,count", [(1, 7), (3, 20 * 500), (8, 256 * 4096 + 13)])
def test_sum_partials_fixed_order(ctx, nparts, count):
    """The library's exchange sum adds the gathered parts in rank order."""
    g = torch.Generator().manual_seed(11 + nparts)
    parts = torch.randn((nparts, count), generator=g, dtype=torch.float64) * torch.logspace(
        0, 12, nparts, dtype=torch.float64)[:, None]
    ref = parts[0].clone()
    for q in range(1, nparts):
        ref = ref + parts[q]
    out = torch.empty(count, dtype=torch.float64, device="cuda")
    assert L.lspca_sum_partials(ctx.handle, parts.cuda(), out) == L.OK
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), ref)

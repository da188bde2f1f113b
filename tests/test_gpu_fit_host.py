"""Host-resident fits (lspca_fit_host): Algorithm 4 over row slices copied from
host memory while the previous slice is computed.

The slices only change the order in which F's terms are summed, so the fit
matches the FP64 oracle within each path's tolerance, and on binary E4M3 X
(integer-exact F per slice) it equals the device-resident fit bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import lspca as O
from oracle import metrics as M
from oracle import philox as P
from paper_1709_07175_gb300 import lspca as L
from paper_1709_07175_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    L.load()
    c = L.Context(0)
    yield c
    c.close()


def _om(w):
    return L.omega("sparse", w.omega_seed, w.p) if w.omega == "sparse" else L.omega("gaussian", w.omega_seed)


@pytest.mark.parametrize("slice_rows", [1000, 0])
def test_fit_host_fp32_matches_oracle_and_device_fit(ctx, slice_rows):
    """FP32 X, very sparse Omega: 3001 rows in slices of 1024 (ragged last
    slice) or one slice; Y within 1e-5 of the oracle (Procrustes-aligned) and
    sigma within 1e-6 of the device-resident fit."""
    w = S.WORKLOADS["fp32_sparse"].scaled(m=3001, n=1024, k=64)
    X = S.generate(w)
    Xh = X.pin_memory()
    r = ctx.fit_host(Xh, w.k, _om(w), slice_rows=slice_rows)
    assert r.status == L.OK and r.report["rank"] == w.k
    rd = ctx.fit(X.cuda(), w.k, _om(w))
    Xd = X.double().numpy()
    fit = O.lspca_fit(Xd, P.omega_sparse(w.omega_seed, w.n, w.k, w.p))
    Y = ctx.project(X.cuda(), r.V).double().cpu().numpy()
    e = M.procrustes_rel(Y, O.project(Xd, fit["V"]))
    assert e < 1e-5, e
    s_h, s_d = r.sigma.cpu().numpy(), rd.sigma.cpu().numpy()
    assert np.max(np.abs(s_h - s_d) / s_d) < 1e-6
    assert np.max(np.abs(s_h - fit["sigma"]) / fit["sigma"]) < 1e-5


def test_fit_host_bf16_gaussian(ctx):
    """BF16 X, Gaussian Omega (BF16-rounded), k = 256, four slices: Y within
    1e-4 of the oracle (the refined low-precision path's tolerance)."""
    w = S.WORKLOADS["bf16_dense"].scaled(m=4001, n=2048)
    X = S.generate(w)
    r = ctx.fit_host(X.pin_memory(), w.k, _om(w), slice_rows=1000)
    Xd = X.double().numpy()
    fit = O.lspca_fit(Xd, P.bf16_rne(P.omega_gaussian(w.omega_seed, w.n, w.k)), route="eig")
    Y = ctx.project(X.cuda(), r.V).double().cpu().numpy()
    e = M.procrustes_rel(Y, O.project(Xd, fit["V"]))
    assert e < 1e-4, e


def test_fit_host_binary_e4m3_equals_device_fit(ctx):
    """Binary E4M3 X with the very sparse Omega: each slice's F is an exact
    integer matrix, so the sliced F equals the unsliced F and the whole fit
    (V and sigma) equals the device-resident fit bit for bit."""
    w = S.WORKLOADS["e4m3_binary"].scaled(m=5001, n=1024, k=128)
    X = S.generate(w)
    r = ctx.fit_host(X.pin_memory(), w.k, _om(w), slice_rows=1200)
    rd = ctx.fit(X.cuda(), w.k, _om(w))
    assert torch.equal(r.V.cpu(), rd.V.cpu())
    assert torch.equal(r.sigma.cpu(), rd.sigma.cpu())


def test_fit_host_pageable_memory(ctx):
    """A pageable (not page-locked) host X gives the same fit as a pinned one."""
    w = S.WORKLOADS["fp32_sparse"].scaled(m=2049, n=512, k=32)
    X = S.generate(w)
    a = ctx.fit_host(X, w.k, _om(w), slice_rows=512)
    b = ctx.fit_host(X.pin_memory(), w.k, _om(w), slice_rows=512)
    assert torch.equal(a.V.cpu(), b.V.cpu())


def test_fit_host_invalid_and_nonfinite(ctx):
    w = S.WORKLOADS["fp32_sparse"].scaled(m=1000, n=256, k=16)
    X = S.generate(w)
    V = torch.empty(w.n, w.k, dtype=torch.float32, device="cuda")
    sig = torch.empty(w.k, dtype=torch.float64, device="cuda")
    # FP64 X is not a host-streaming type
    assert L.lspca_fit_host(ctx.handle, X.double(), w.k, _om(w), 0, 0, V, sig) == L.ERR_INVALID
    # k not a multiple of 4
    assert L.lspca_fit_host(ctx.handle, X, 15, _om(w), 0, 0, V, sig) == L.ERR_INVALID
    # the Gram is not produced here
    assert L.lspca_fit_host(ctx.handle, X, w.k, _om(w), L.WANT_GRAM, 0, V, sig) == L.ERR_INVALID
    # NaN in the last slice
    Xn = X.clone()
    Xn[900, 7] = float("nan")
    rep = L.lspca_report()
    rc = L.lspca_fit_host(ctx.handle, Xn.pin_memory(), w.k, _om(w), 0, 256, V, sig, None, None, rep)
    assert rc == L.ERR_NUMERIC
    assert ctx.sync_status() == L.OK


@pytest.mark.parametrize("wname,m,n,k,slice_rows", [("e4m3_binary", 300_001, 512, 256, 65_536),
                                                    ("bf16_dense", 20_000, 1024, 64, 6_000),
                                                    ("fp32_sparse", 5_000, 1024, 128, 2_048)])
def test_fit_project_host(ctx, wname, m, n, k, slice_rows):
    """lspca_fit_project_host: the fit equals lspca_fit_host's bit for bit (the
    same slices and kernels), X lands in the device buffer unchanged, and Y
    (projected in slices of about 128 MB and copied back while the next slice
    runs; three slices with a ragged last one at k = 256) matches the
    reduction map of the whole resident X within 1e-6 of its norm."""
    w = S.WORKLOADS[wname].scaled(m=m, n=n, k=k)
    X = S.generate(w)
    Xh = X.pin_memory()
    om = _om(w)
    ref = ctx.fit_host(Xh, w.k, om, slice_rows=slice_rows)
    Xd = torch.empty(X.shape, dtype=X.dtype, device="cuda")
    V = torch.empty(n, k, dtype=torch.float32, device="cuda")
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    rk = torch.empty(1, dtype=torch.int32, device="cuda")
    Yh = torch.full((m, k), float("nan"), dtype=torch.float32).pin_memory()
    rep = L.lspca_report()
    rc = L.lspca_fit_project_host(ctx.handle, Xh, k, om, 0, slice_rows, Xd, V, sig, Yh, rk, report=rep)
    assert rc == L.OK, L.lspca_strerror(rc)
    torch.cuda.synchronize()
    assert torch.equal(Xd.cpu().view(torch.uint8), X.view(torch.uint8))
    assert torch.equal(V, ref.V) and torch.equal(sig, ref.sigma)
    Yd = ctx.project(Xd, V)
    torch.cuda.synchronize()
    Yd = Yd.cpu()
    assert torch.isfinite(Yh).all()
    rel = ((Yh.double() - Yd.double()).norm() / Yd.double().norm()).item()
    assert rel < 1e-6, rel
    assert L.lspca_fit_project_host(ctx.handle, Xh, k, om, 0, slice_rows, None, V, sig, Yh, rk) == L.ERR_INVALID

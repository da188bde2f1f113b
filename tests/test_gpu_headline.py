"""GPU parity at the shapes of the headline workloads and on a steep spectrum.

* Binary features in FP8 E4M3 at n = 4,096, k = 256 with the very sparse
  Omega (p = 64), the shape of the paper-scale workload (Experiment 1's
  mostly-binary design matrix) at m = 20,000 rows: U = X Omega and
  F = U^T X are integers and must equal the oracle's products bit for bit;
  the fit's reduced data within 1e-4 (refined low-precision path).
* BF16 X at n = 8,192, k = 256 with the Gaussian Omega (the precision
  workload's shape) on a 20,000-row sample: reduced data and sigma within 1e-4.
* sigma_i = 2^-i (FP64 path, k = 64 and 256): the eigenvalues of F F^T span
  the whole FP64 range; sigma, the subspaces and the rank against the oracle.

Where singular values are well separated (relative gap above 1e-2) the columns
of the reduced data are compared one by one after sign alignment.
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
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_07175_gb300 import build
    build.build()
    c = L.Context(0)
    yield c
    c.close()


def _separated(sigma, tol=1e-2):
    s = np.asarray(sigma, np.float64)
    gap = np.minimum(np.r_[np.inf, -np.diff(s)], np.r_[-np.diff(s), np.inf]) / np.maximum(s, 1e-300)
    return gap > tol


def _column_errors(Y, Yref, cols):
    """Relative error of each selected column after sign alignment."""
    out = []
    for j in np.nonzero(cols)[0]:
        a, b = Y[:, j], Yref[:, j]
        sgn = 1.0 if a @ b >= 0 else -1.0
        out.append(np.linalg.norm(sgn * a - b) / max(np.linalg.norm(b), 1e-300))
    return np.array(out)


C4H = S.WORKLOADS["e4m3_binary"].scaled(m=20000)       # n = 4096, k = 256, p = 64
C3H = S.WORKLOADS["bf16_dense"].scaled(m=20000)        # n = 8192, k = 256, Gaussian Omega


@pytest.fixture(scope="module")
def c4():
    w = C4H
    X = S.generate(w)
    Xd = X.float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    fit = O.lspca_fit(Xd, Om, route="eig")
    return w, X, Xd, Om, fit


def test_c4_shape_sketch_and_chain_bit_exact(ctx, c4):
    w, X, Xd, Om, fit = c4
    assert (w.n, w.k, w.p) == (4096, 256, 64)
    Uref = O.sketch(Xd, Om)
    Fref = O.chain(Uref, Xd)
    assert np.abs(Fref).max() < 2 ** 24 and np.array_equal(Uref, np.round(Uref))
    Xg = X.cuda()
    U = ctx.sketch(Xg, w.k, L.omega("sparse", w.omega_seed, w.p))
    assert np.array_equal(U.double().cpu().numpy(), Uref)
    F, _ = ctx.chain(Xg, U)
    assert np.array_equal(F.cpu().numpy(), Fref)


def test_c4_shape_fit(ctx, c4):
    w, X, Xd, Om, fit = c4
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, L.omega("sparse", w.omega_seed, w.p))
    assert r.status == L.OK and r.report["rank"] == fit["rank"] == w.k
    sig = r.sigma.cpu().numpy()
    assert np.max(np.abs(sig - fit["sigma"]) / fit["sigma"]) < 1e-6
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    assert M.procrustes_rel(Y, Yref) < 1e-4
    cols = _separated(fit["sigma"])
    assert cols.sum() >= 8
    ce = _column_errors(Y, Yref, cols)
    print("c4 shape: separated columns", int(cols.sum()), "max column error", ce.max())
    assert ce.max() < 1e-4


def test_c3_shape_fit_on_sample(ctx):
    w = C3H
    assert (w.n, w.k) == (8192, 256)
    X = S.generate(w)
    Xd = X.double().numpy()
    Om = P.bf16_rne(P.omega_gaussian(w.omega_seed, w.n, w.k))
    fit = O.lspca_fit(Xd, Om, route="eig")
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, L.omega("gaussian", w.omega_seed))
    sig = r.sigma.cpu().numpy()
    assert np.max(np.abs(sig - fit["sigma"]) / fit["sigma"]) < 1e-4
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    assert M.procrustes_rel(Y, Yref) < 1e-4
    cols = _separated(fit["sigma"])
    ce = _column_errors(Y, Yref, cols)
    print("c3 shape: separated columns", int(cols.sum()), "max column error", ce.max() if ce.size else None)
    if ce.size:
        assert ce.max() < 1e-4


@pytest.mark.parametrize("k", [64, 256])
def test_steep_spectrum_fit(ctx, k):
    w = S.STEEP.scaled(k=k, n=1000 if k == 64 else 1200)
    X = S.generate(w)
    Xd = X.numpy()
    Om = P.omega_gaussian(w.omega_seed, w.n, w.k)
    fit = O.lspca_fit(Xd, Om, route="eig")
    r = ctx.fit(X.cuda(), w.k, L.omega("gaussian", w.omega_seed))
    rank = int(r.rank.item())
    assert abs(rank - fit["rank"]) <= 1
    sig = r.sigma.cpu().numpy()
    big = fit["sigma"] > 1e-4 * fit["sigma"][0]      # decades the eigen route keeps accurate
    assert big.sum() >= 6
    assert np.max(np.abs(sig[big] - fit["sigma"][big]) / fit["sigma"][big]) < 1e-8
    V = r.V.cpu().numpy()
    nb = int(big.sum())
    assert M.max_sine(fit["V"][:, :nb], V[:, :nb]) < 1e-8
    Y = O.project(Xd, V)
    Yref = O.project(Xd, fit["V"])
    # both sides take the eigen route, whose eigenvectors for lambda_i ~ 1e-12
    # lambda_1 carry ~eps lambda_1 / gap ~ 1e-4 of FP64 noise of their own;
    # weighted by their sigma that bounds the difference of the reduced data
    assert M.procrustes_rel(Y, Yref) < 1e-7
    ce = _column_errors(Y, Yref, big & _separated(fit["sigma"]))
    assert ce.max() < 1e-8


@pytest.mark.parametrize("k", [64, 256])
def test_steep_spectrum_k_by_k_step_time_is_bounded(ctx, k):
    """The k x k step on sigma(F) = 2^-i takes milliseconds, not hundreds of them."""
    n = 4096
    rng = np.random.default_rng(k)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    Pm, _ = np.linalg.qr(rng.standard_normal((k, k)))
    F = torch.from_numpy((Pm * 2.0 ** -np.arange(1, k + 1.0)) @ Q.T).cuda().contiguous()
    ctx.decompose(F, 200000, torch.float32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        ctx.decompose(F, 200000, torch.float32)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    print(f"k = {k}: k x k step {ms:.2f} ms")
    assert ms < 20.0

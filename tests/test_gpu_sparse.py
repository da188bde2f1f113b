"""Sparse X in CSR form (lspca_fit_csr, lspca_project_csr) against the FP64
oracle's sparse fit (the definitions of Algorithm 2 with sparse-dense matrix
products), on seeded TF-IDF-shaped inputs."""
import numpy as np
import pytest
import torch

from oracle import lspca as O
from oracle import metrics as M
from oracle import philox as P
from paper_1709_07175_gb300 import lspca as L
from paper_1709_07175_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
sp = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def ctx():
    L.load()
    c = L.Context(0)
    yield c
    c.close()


def _csr(m, n, density, seed):
    rp, c, v = S.sparse_csr(m, n, density, seed)
    Xs = sp.csr_matrix((v.numpy(), c.numpy(), rp.numpy()), shape=(m, n))
    return (rp.cuda(), c.cuda(), v.cuda()), Xs


def _om(kind, seed, n, k, p):
    if kind == "gaussian":
        return P.omega_gaussian(seed, n, k), L.omega("gaussian", seed)
    return P.omega_sparse(seed, n, k, p), L.omega("sparse", seed, p)


@pytest.mark.parametrize("kind", ["sparse", "gaussian"])
def test_fit_csr_matches_oracle(ctx, kind):
    """3,000 x 2,000 at density 0.005, k = 32: Y (by lspca_project_csr) within
    1e-5 of the oracle's (Procrustes-aligned), sigma within 1e-5."""
    (rp, c, v), Xs = _csr(3000, 2000, 0.005, seed=11)
    Om, om = _om(kind, 3, 2000, 32, 45)
    r = ctx.fit_csr(rp, c, v, 2000, 32, om)
    assert r.status == L.OK and r.report["rank"] == 32
    fit = O.lspca_fit_sparse(Xs, Om)
    Y = ctx.project_csr(rp, c, v, 2000, r.V).double().cpu().numpy()
    Yref = np.asarray(Xs.astype(np.float64) @ fit["V"])
    assert M.procrustes_rel(Y, Yref) < 1e-5
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-5


def test_fit_csr_tfidf_shape(ctx):
    """The TF-IDF shape (74,067 x 28,606, density 0.000513, ~1.09 M nonzeros,
    heavy head columns), k = 128, very sparse Omega p = 169: Y within 1e-5 of
    the oracle (Procrustes-aligned), sigma within 1e-5; two fits are
    bit-identical."""
    w = S.SPARSE_TFIDF
    (rp, c, v), Xs = _csr(w["m"], w["n"], w["density"], w["seed"])
    Om, om = _om("sparse", w["omega_seed"], w["n"], w["k"], w["p"])
    r = ctx.fit_csr(rp, c, v, w["n"], w["k"], om)
    assert r.status == L.OK
    r2 = ctx.fit_csr(rp, c, v, w["n"], w["k"], om)
    assert torch.equal(r.V, r2.V) and torch.equal(r.sigma, r2.sigma)
    fit = O.lspca_fit_sparse(Xs, Om)
    Y = ctx.project_csr(rp, c, v, w["n"], r.V).double().cpu().numpy()
    Yref = np.asarray(Xs.astype(np.float64) @ fit["V"])
    assert M.procrustes_rel(Y, Yref) < 1e-5
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-5


def test_project_csr_equals_dense_product(ctx):
    """Y = X V for CSR X (with empty rows) equals the FP64 product to FP32 rounding."""
    (rp, c, v), Xs = _csr(1500, 700, 0.01, seed=12)
    rp_h = rp.cpu().numpy().copy()
    keep = np.ones(1500, bool)
    keep[::7] = False  # empty every seventh row
    rows = [np.arange(rp_h[i], rp_h[i + 1]) for i in range(1500) if keep[i]]
    cnt = np.array([rp_h[i + 1] - rp_h[i] if keep[i] else 0 for i in range(1500)])
    idx = np.concatenate(rows)
    rp2 = torch.from_numpy(np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)).cuda()
    c2 = c[torch.from_numpy(idx).cuda()].contiguous()
    v2 = v[torch.from_numpy(idx).cuda()].contiguous()
    X2 = sp.csr_matrix((v2.cpu().numpy(), c2.cpu().numpy(), rp2.cpu().numpy()), shape=(1500, 700))
    V = torch.randn(700, 48, generator=torch.Generator().manual_seed(3)).cuda()
    Y = ctx.project_csr(rp2, c2, v2, 700, V).double().cpu().numpy()
    Yref = np.asarray(X2.astype(np.float64) @ V.double().cpu().numpy())
    assert np.all(Y[~keep] == 0)
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < 1e-7


def test_csr_bad_index_and_nonfinite(ctx):
    (rp, c, v), _ = _csr(800, 300, 0.02, seed=13)
    om = L.omega("sparse", 0, 17)
    V = torch.empty(300, 16, device="cuda")
    sig = torch.empty(16, dtype=torch.float64, device="cuda")
    # a column index out of range: reported, nothing written out of bounds
    cb = c.clone()
    cb[5] = 300
    rep = L.lspca_report()
    assert L.lspca_fit_csr(ctx.handle, rp, cb, v, 300, 16, om, 0, V, sig, None, None, rep) == L.ERR_INVALID
    assert ctx.sync_status() == L.OK
    # a NaN value
    vn = v.clone()
    vn[9] = float("nan")
    rep = L.lspca_report()
    assert L.lspca_fit_csr(ctx.handle, rp, c, vn, 300, 16, om, 0, V, sig, None, None, rep) == L.ERR_NUMERIC
    assert ctx.sync_status() == L.OK
    # invalid arguments
    assert L.lspca_fit_csr(ctx.handle, rp, c, v, 300, 301, om, 0, V, sig) == L.ERR_INVALID  # k > n
    assert L.lspca_fit_csr(ctx.handle, rp, c, v, 300, 16, om, L.WANT_GRAM, V, sig) == L.ERR_INVALID

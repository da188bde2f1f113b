"""Parity at the benchmarked size: fp32_sparse, X 200,000 x 4,096 FP32, k = 128,
very sparse Omega (p = 64), in the launch configuration bench.py times.

The FP64 oracle runs the whole fit at full size (two 1e11-flop products and
the k x k step), and the GPU result is compared on:
* the singular values sigma~ (relative 1e-5);
* the subspace of V (largest principal-angle sine 1e-4) and its orthonormality;
* 2,000 sampled rows of U = X Omega (FP32 gather bound, as the small tests);
* the reduced data Y = X V on 20,000 sampled rows (relative Frobenius 1e-5,
  Procrustes-aligned, as the small tests).
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
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_07175_gb300 import build
    build.build()
    w = S.WORKLOADS["fp32_sparse"]
    X = S.generate(w)  # CPU generation (FP64 factors), stored FP32
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    Xd = X.numpy().astype(np.float64)
    U = Xd @ Om
    F = U.T @ Xd
    Vref, sref, rref = O.decompose_eig(F, w.m, w.n)
    ctx = L.Context(0)
    yield w, X, Xd, Om, U, Vref, sref, ctx
    ctx.close()


def test_fullsize_fit_parity(setup):
    w, X, Xd, Om, U, Vref, sref, ctx = setup
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, L.omega("sparse", w.omega_seed, w.p))
    assert r.status == L.OK
    V = r.V.double().cpu().numpy()
    sig = r.sigma.cpu().numpy()
    srel = np.max(np.abs(sig - sref) / sref)
    sine = M.max_sine(Vref, V)
    orth = np.abs(V.T @ V - np.eye(w.k)).max()
    rng = np.random.default_rng(123)
    rows = np.sort(rng.choice(w.m, 20000, replace=False))
    Xs = X[rows].cuda()
    Y = ctx.project(Xs, r.V).double().cpu().numpy()
    Yref = Xd[rows] @ Vref
    pr = M.procrustes_rel(Y, Yref)
    print(f"fullsize: sigma rel {srel:.2e} sine {sine:.2e} orth {orth:.2e} Y procrustes {pr:.2e} "
          f"signaligned {M.signaligned_rel(Y, Yref):.2e}")
    assert srel < 1e-5
    assert sine < 1e-4
    assert orth < 1e-6
    assert pr < 1e-5


def test_fullsize_sketch_rows(setup):
    w, X, Xd, Om, U, Vref, sref, ctx = setup
    Ug = ctx.sketch(X.cuda(), w.k, L.omega("sparse", w.omega_seed, w.p))
    rng = np.random.default_rng(7)
    rows = rng.choice(w.m, 2000, replace=False)
    got = Ug[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    ref = U[rows]
    bound = (np.abs(Xd[rows]) @ np.abs(Om)) * (np.count_nonzero(Om, axis=0) * 2.0 ** -24) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)

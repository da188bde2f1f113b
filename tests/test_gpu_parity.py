"""GPU parity: the CUDA library, called through its C ABI, against the FP64 oracle.

Both sides consume the same seeded inputs (paper_1709_07175_gb300.synthetic);
each side generates Omega itself (Philox4x32-10 from its published
definition).  Tolerances (written in each test):

* Omega: very sparse bit-exact; Gaussian within 1 FP32 ulp.
* FP64 path (workload fp64_small): reduced data Y within 1e-10 (relative
  Frobenius, Procrustes-aligned), sigma within 1e-10 relative.
* FP32 path (fp32_sparse at reduced m): Y within 1e-5 (Procrustes-aligned).
  The reduced data is unique only up to an orthogonal k x k factor when
  singular values nearly coincide (Prop. 3 and the footnote of Sec. III-B.2),
  so the binding comparison aligns with the orthogonal Procrustes factor;
  the per-column sign-aligned error and the subspace sine are reported.
"""
import math

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


def _omega_np(w):
    if w.omega == "gaussian":
        return P.omega_gaussian(w.omega_seed, w.n, w.k)
    return P.omega_sparse(w.omega_seed, w.n, w.k, w.p)


def _om(w):
    return L.omega(w.omega, w.omega_seed, w.p)


C1 = S.WORKLOADS["fp64_small"]
C2S = S.WORKLOADS["fp32_sparse"].scaled(m=3001)          # 94 row tiles, ragged tail
C2R = S.WORKLOADS["fp32_sparse"].scaled(m=2049, n=1000)   # ragged chunk and ragged rows


@pytest.fixture(scope="module")
def data():
    out = {}
    for w in (C1, C2S, C2R):
        X = S.generate(w)
        Om = _omega_np(w)
        Xd = X.double().numpy()
        fit = O.lspca_fit(Xd, Om, route="eig")
        out[w.name + str(w.m) + "x" + str(w.n)] = (w, X, Xd, Om, fit)
    return out


def _get(data, w):
    return data[w.name + str(w.m) + "x" + str(w.n)]


# ------------------------------------------------------------------ Omega

@pytest.mark.parametrize("n,k,p,seed", [(4096, 128, 64, 0), (1000, 37, 3, 12345678901), (513, 256, 64, 7)])
def test_sparse_omega_bit_exact(ctx, n, k, p, seed):
    om = L.omega("sparse", seed, p)
    g = ctx.omega(om, n, k, torch.float64).cpu().numpy()
    ref = P.omega_sparse(seed, n, k, p)
    assert np.array_equal(g, ref)


@pytest.mark.parametrize("n,k,seed", [(8192, 256, 0), (500, 20, 0), (77, 9, 2 ** 40 + 3)])
def test_gaussian_omega_within_one_ulp(ctx, n, k, seed):
    om = L.omega("gaussian", seed)
    g = ctx.omega(om, n, k, torch.float32).cpu().numpy()
    ref = P.omega_gaussian(seed, n, k).astype(np.float32)
    gi = g.view(np.int32).astype(np.int64)
    ri = ref.view(np.int32).astype(np.int64)
    assert np.max(np.abs(gi - ri)) <= 1
    # the BF16 form is the round-to-nearest-even of the FP32 value
    gb = ctx.omega(om, n, k, torch.bfloat16).float().cpu().numpy()
    assert np.array_equal(gb, torch.from_numpy(g).to(torch.bfloat16).float().numpy())


# ------------------------------------------------------------------ pass S

def test_sketch_fp64(ctx, data):
    w, X, Xd, Om, fit = _get(data, C1)
    U = ctx.sketch(X.cuda(), w.k, _om(w)).cpu().numpy()
    ref = fit["U"]
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("wl", [C2S, C2R])
def test_sketch_sparse_fp32(ctx, data, wl):
    w, X, Xd, Om, fit = _get(data, wl)
    U = ctx.sketch(X.cuda(), w.k, _om(w)).double().cpu().numpy()
    ref = fit["U"]
    # sequential FP32 sum of the nnz_c signed terms: |err| <= nnz_c u sum|terms|
    bound = (np.abs(Xd) @ np.abs(Om)) * (np.count_nonzero(Om, axis=0) * 2.0 ** -24) + 1e-30
    assert np.all(np.abs(U - ref) <= bound)


@pytest.mark.parametrize("dtype,m,n,ldx,k", [(torch.float32, 777, 1001, 1004, 64),
                                             (torch.float32, 300, 4096, 4096, 128),
                                             (torch.float32, 1100, 1000, 1000, 64),
                                             (torch.float32, 515, 2040, 2056, 100),
                                             (torch.float32, 1, 1000, 1000, 64),
                                             (torch.float32, 100, 4096, 4096, 128),
                                             (torch.bfloat16, 515, 1003, 1008, 100),
                                             (torch.bfloat16, 129, 2048, 2048, 128)])
def test_sketch_sparse_strided_and_ragged(ctx, dtype, m, n, ldx, k):
    """Pass S of the very sparse Omega on FP32 / BF16 X with ragged row tiles,
    a ragged last column step (n not a multiple of the copy width, X rows
    padded to ldx) and k not a multiple of 16: the FP32 gather sum is within
    the sequential-summation bound of the FP64 oracle.  The FP32 cases with n
    and ldx multiples of 8 run the kernel that keeps its A operand in tensor
    memory (k = 64: one 64-column N tile; k = 100: two), the others the
    shared-memory one."""
    w = S.WORKLOADS["fp32_sparse"].scaled(m=m, n=ldx, k=k)
    base = S.generate(w).to(dtype)
    X = base.cuda()[:, :n]  # row-strided view, ldx > n where the two differ
    Xd = base[:, :n].double().numpy()
    Om = P.omega_sparse(w.omega_seed, n, k, w.p)
    U = ctx.sketch(X, k, L.omega("sparse", w.omega_seed, w.p)).double().cpu().numpy()
    ref = O.sketch(Xd, Om)
    bound = (np.abs(Xd) @ np.abs(Om)) * (np.count_nonzero(Om, axis=0) * 2.0 ** -24) + 1e-30
    assert np.all(np.abs(U - ref) <= bound)


# ------------------------------------------------------------------ pass F

def test_chain_fp64(ctx, data):
    w, X, Xd, Om, fit = _get(data, C1)
    U = torch.from_numpy(fit["U"]).cuda()
    F, G = ctx.chain(X.cuda(), U, want_gram=True)
    F = F.cpu().numpy()
    G = G.cpu().numpy()
    assert np.linalg.norm(F - fit["F"]) / np.linalg.norm(fit["F"]) < 1e-13
    assert np.linalg.norm(G - fit["G"]) / np.linalg.norm(fit["G"]) < 1e-13


@pytest.mark.parametrize("wl", [C2S, C2R])
def test_chain_fp32(ctx, data, wl):
    w, X, Xd, Om, fit = _get(data, wl)
    U32 = torch.from_numpy(fit["U"]).float()
    Ud = U32.double().numpy()
    F, G = ctx.chain(X.cuda(), U32.cuda(), want_gram=True)
    Fref = Ud.T @ Xd
    Gref = Ud.T @ Ud
    # FP32 accumulation within a split, FP64 across splits
    assert np.linalg.norm(F.cpu().numpy() - Fref) / np.linalg.norm(Fref) < 2e-6
    assert np.linalg.norm(G.cpu().numpy() - Gref) / np.linalg.norm(Gref) < 2e-6


@pytest.mark.parametrize("dtype,m,n,ldx,k", [("f32", 3001, 1000, 1000, 100), ("f32", 2049, 4096, 4096, 256),
                                             ("f32", 777, 1001, 1004, 20), ("bf16", 3001, 1000, 1000, 100),
                                             ("bf16", 1025, 2048, 2056, 200), ("e4m3", 1500, 1040, 1040, 64),
                                             ("e4m3", 700, 4096, 4096, 256)])
def test_chain_tensor_core_paths(ctx, dtype, m, n, ldx, k):
    """Pass F (F = U^T X with G = U^T U) on every tensor-core path, with a ragged
    row tail, a partial last column tile, k below one 128-row half or spanning
    two, and row-strided X.  Against the FP64 products of the same stored
    values (relative Frobenius): FP32 X with split-FP16 operands 2e-6; BF16 and
    E4M3 X (exact) with a split-BF16 U 2e-5; G from FP16 pairs of U 2e-6."""
    if dtype == "e4m3":
        w = S.WORKLOADS["e4m3_binary"].scaled(m=m, n=ldx, k=k)
    elif dtype == "bf16":
        w = S.WORKLOADS["bf16_dense"].scaled(m=m, n=ldx, k=k)
    else:
        w = S.WORKLOADS["fp32_sparse"].scaled(m=m, n=ldx, k=k)
    base = S.generate(w)
    X = base.cuda()[:, :n]
    Xd = base[:, :n].float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, n, k, 64)
    U32 = torch.from_numpy(Xd @ Om).float()
    Ud = U32.double().numpy()
    F, G = ctx.chain(X, U32.cuda(), want_gram=True)
    Fref = Ud.T @ Xd
    Gref = Ud.T @ Ud
    ef = np.linalg.norm(F.cpu().numpy() - Fref) / np.linalg.norm(Fref)
    eg = np.linalg.norm(G.cpu().numpy() - Gref) / np.linalg.norm(Gref)
    assert ef < (2e-6 if dtype == "f32" else 2e-5), ef
    assert eg < 2e-6, eg


# ------------------------------------------------------------------ the k x k step

@pytest.mark.parametrize("wl", [C1, C2S])
def test_decompose_matches_oracle_eig_route(ctx, data, wl):
    w, X, Xd, Om, fit = _get(data, wl)
    F = torch.from_numpy(fit["F"]).cuda()
    V, sigma, rank = ctx.decompose(F, w.m, torch.float64)
    V = V.cpu().numpy()
    sigma = sigma.cpu().numpy()
    assert int(rank.item()) == fit["rank"] == w.k
    assert np.max(np.abs(sigma - fit["sigma"]) / fit["sigma"]) < 1e-11
    assert np.abs(V.T @ V - np.eye(w.k)).max() < 1e-11
    assert M.max_sine(fit["V"], V) < 1e-10
    # columns with a clear gap agree individually (sign rule applied on both sides)
    s = fit["sigma"]
    gap = np.minimum(np.r_[np.inf, -np.diff(s)], np.r_[-np.diff(s), np.inf]) / s[0]
    sep = gap > 1e-3
    assert np.abs(V[:, sep] - fit["V"][:, sep]).max() < 1e-8


# ------------------------------------------------------------------ full fits

def _report_errors(Y, Yref, V, Vref):
    return {"procrustes": M.procrustes_rel(Y, Yref), "signaligned": M.signaligned_rel(Y, Yref),
            "sine": M.max_sine(Vref, V), "chordal": M.chordal(Vref, V)}


def test_fit_fp64_parity(ctx, data):
    w, X, Xd, Om, fit = _get(data, C1)
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, _om(w))
    assert r.status == L.OK and r.report["rank"] == w.k
    V = r.V.cpu().numpy()
    Y = ctx.project(Xg, r.V).cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    e = _report_errors(Y, Yref, V, fit["V"])
    print("fp64_small", e)
    assert e["procrustes"] < 1e-10
    assert e["sine"] < 1e-10
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-10
    # the FP64 path has well separated singular values: per-column agreement too
    assert e["signaligned"] < 1e-8


@pytest.mark.parametrize("wl", [C2S, C2R])
def test_fit_fp32_parity(ctx, data, wl):
    w, X, Xd, Om, fit = _get(data, wl)
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, _om(w))
    assert r.status == L.OK
    V = r.V.double().cpu().numpy()
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    e = _report_errors(Y, Yref, V, fit["V"])
    print(w.name, w.m, w.n, e)
    assert e["procrustes"] < 1e-5
    assert e["sine"] < 1e-4
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-5


def test_fit_fp32_gaussian_parity(ctx):
    """FP32 X with the Gaussian Omega: the sketch takes Omega in three exact
    BF16 pieces (six products, A in tensor memory).  U within 2e-6 of the FP64
    product of the same stored values (relative Frobenius); the fit's Y within
    1e-5 of the oracle's (Procrustes-aligned) and sigma within 1e-5."""
    w = S.WORKLOADS["fp32_sparse"].scaled(m=3001, n=1024, k=64)
    X = S.generate(w)
    Xd = X.double().numpy()
    Om = P.omega_gaussian(7, w.n, w.k)  # FP64 draws rounded to FP32, as the library stores them
    om = L.omega("gaussian", 7)
    U = ctx.sketch(X.cuda(), w.k, om).double().cpu().numpy()
    Uref = Xd @ Om
    assert np.linalg.norm(U - Uref) / np.linalg.norm(Uref) < 2e-6
    r = ctx.fit(X.cuda(), w.k, om)
    assert r.status == L.OK
    fit = O.lspca_fit(Xd, Om)
    Y = ctx.project(X.cuda(), r.V).double().cpu().numpy()
    assert M.procrustes_rel(Y, O.project(Xd, fit["V"])) < 1e-5
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-5


@pytest.mark.parametrize("kind", ["gaussian", "sparse"])
def test_fit_oversampled_parity(ctx, kind):
    """Oversampled fit (l = 44 > k = 32, FP32 X): the top k of the l-column fit.
    Y within 1e-5 of the oracle's (Procrustes-aligned), sigma within 1e-5,
    rank k; and l = k gives lspca_fit's result bit for bit."""
    w = S.WORKLOADS["fp32_sparse"].scaled(m=3001, n=1024, k=32)
    X = S.generate(w)
    Xd = X.double().numpy()
    l = 44
    if kind == "gaussian":
        Om, om = P.omega_gaussian(7, w.n, l), L.omega("gaussian", 7)
    else:
        Om, om = P.omega_sparse(7, w.n, l, w.p), L.omega("sparse", 7, w.p)
    r = ctx.fit_oversampled(X.cuda(), w.k, l, om)
    assert r.status == L.OK and int(r.rank.item()) == w.k and r.report["rank"] == w.k
    fit = O.lspca_fit_oversampled(Xd, Om, w.k)
    Y = ctx.project(X.cuda(), r.V).double().cpu().numpy()
    assert M.procrustes_rel(Y, O.project(Xd, fit["V"])) < 1e-5
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-5
    same = ctx.fit_oversampled(X.cuda(), w.k, w.k, om)
    plain = ctx.fit(X.cuda(), w.k, om)
    assert torch.equal(same.V, plain.V) and torch.equal(same.sigma, plain.sigma)


def test_fit_is_deterministic(ctx, data):
    w, X, Xd, Om, fit = _get(data, C2S)
    Xg = X.cuda()
    a = ctx.fit(Xg, w.k, _om(w))
    b = ctx.fit(Xg, w.k, _om(w))
    assert torch.equal(a.V, b.V) and torch.equal(a.sigma, b.sigma)


def test_force_simt_agrees(ctx, data):
    w, X, Xd, Om, fit = _get(data, C2S)
    Xg = X.cuda()
    a = ctx.fit(Xg, w.k, _om(w))
    b = ctx.fit(Xg, w.k, _om(w), flags=L.FORCE_SIMT)
    Ya = ctx.project(Xg, a.V).double().cpu().numpy()
    Yb = ctx.project(Xg, b.V).double().cpu().numpy()
    assert M.procrustes_rel(Ya, Yb) < 1e-5


# ------------------------------------------------------------------ SPCA path

def test_spca_fp64_parity_and_prop2(ctx, data):
    w, X, Xd, Om, fit = _get(data, C1)
    Xg = X.cuda()
    sp = O.spca_fit(Xd, Om, route="eig")
    r = ctx.spca(Xg, w.k, _om(w))
    Vs = r.V.cpu().numpy()
    assert M.max_sine(sp["V"], Vs) < 1e-10
    assert np.max(np.abs(r.sigma.cpu().numpy() - sp["sigma"]) / sp["sigma"]) < 1e-9
    # Prop. 2 on the GPU: V^s and V^l span the same subspace
    rl = ctx.fit(Xg, w.k, _om(w))
    assert M.max_sine(rl.V.cpu().numpy(), Vs) < 1e-10
    # Prop. 3: equal pairwise distances in the reduced space
    Ys = ctx.project(Xg, r.V).cpu().numpy()
    Yl = ctx.project(Xg, rl.V).cpu().numpy()
    rng = np.random.default_rng(0)
    i, j = rng.integers(0, w.m, 2000), rng.integers(0, w.m, 2000)
    keep = i != j
    ds = np.linalg.norm(Ys[i[keep]] - Ys[j[keep]], axis=1)
    dl = np.linalg.norm(Yl[i[keep]] - Yl[j[keep]], axis=1)
    assert np.max(np.abs(ds - dl) / dl) < 1e-10


def test_spca_fp32_parity(ctx, data):
    w, X, Xd, Om, fit = _get(data, C2S)
    Xg = X.cuda()
    sp = O.spca_fit(Xd, Om, route="eig")
    r = ctx.spca(Xg, w.k, _om(w))
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, sp["V"])
    assert M.procrustes_rel(Y, Yref) < 1e-5
    assert np.max(np.abs(r.sigma.cpu().numpy() - sp["sigma"]) / sp["sigma"]) < 1e-4


@pytest.mark.parametrize("wl", [C2S, C2R])
def test_spca_cholesky_qr2_agrees_with_householder_and_oracle(ctx, data, wl):
    """SPCA's R by CholeskyQR2 (tensor-core path) and by the Householder TSQR
    (the SIMT path, LSPCA_FORCE_SIMT): the same span (Prop. 2 holds for any
    invertible R, and both equal Lazy SPCA's), singular values of Q^T X within
    1e-4 of the oracle for both, and within 2e-5 of each other."""
    w, X, Xd, Om, fit = _get(data, wl)
    Xg = X.cuda()
    sp = O.spca_fit(Xd, Om, route="eig")
    cq = ctx.spca(Xg, w.k, _om(w))
    hh = ctx.spca(Xg, w.k, _om(w), flags=L.FORCE_SIMT)
    assert cq.report["qr_path"] == 1 and hh.report["qr_path"] == 2
    s_cq, s_hh = cq.sigma.cpu().numpy(), hh.sigma.cpu().numpy()
    e_cq = np.max(np.abs(s_cq - sp["sigma"]) / sp["sigma"])
    e_hh = np.max(np.abs(s_hh - sp["sigma"]) / sp["sigma"])
    print(f"SPCA sigma vs oracle: CholeskyQR2 {e_cq:.2e}, Householder {e_hh:.2e}")
    assert e_cq < 1e-4 and e_hh < 1e-4
    assert np.max(np.abs(s_cq - s_hh) / s_hh) < 2e-5
    assert M.max_sine(cq.V.double().cpu().numpy(), hh.V.double().cpu().numpy()) < 1e-4
    assert M.max_sine(cq.V.double().cpu().numpy(), sp["V"]) < 1e-4


def test_spca_falls_back_to_householder_on_rank_deficient_u(ctx):
    """An X of rank 5 (up to its FP32 rounding) sketched to k = 16: U^T U is
    singular to working precision, the first Cholesky stops, and the
    Householder TSQR gives R; R^-T F drops the directions whose pivots are
    below 1e-4 of the largest (dividing F's rounding error by them took the
    rank to k and buried the signal), and the fit recovers the rank-5
    subspace exactly."""
    X, B = S.rank_r_exact(4000, 1000, 5, seed=3)
    Xg = X.float().cuda()
    r = ctx.spca(Xg, 16, L.omega("gaussian", 9))
    assert r.report["qr_path"] == 2
    V = r.V.double().cpu().numpy()
    assert np.all(np.isfinite(V)) and np.all(np.isfinite(r.sigma.cpu().numpy()))
    assert int(r.rank.item()) == 5
    assert M.max_sine(B.numpy(), V[:, :5]) < 1e-4


# ------------------------------------------------------------------ projection

@pytest.mark.parametrize("wl,tol", [(C1, 1e-13), (C2S, 2e-6), (C2R, 2e-6)])
def test_project_matches_oracle(ctx, data, wl, tol):
    w, X, Xd, Om, fit = _get(data, wl)
    rt = torch.float64 if w.dtype == "f64" else torch.float32
    V = torch.from_numpy(fit["V"]).to(rt)
    Y = ctx.project(X.cuda(), V.cuda()).double().cpu().numpy()
    Yref = Xd @ V.double().numpy()
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < tol


# ------------------------------------------------------------------ edge cases

def test_rank_deficient_input(ctx):
    X, B = S.rank_r_exact(4000, 1000, 5, seed=3)
    Xg = X.cuda()
    r = ctx.fit(Xg, 8, L.omega("gaussian", 9))
    assert r.status == L.WARN_RANK_DEFICIENT
    assert r.report["rank"] == 5 and int(r.rank.item()) == 5
    V = r.V.cpu().numpy()
    assert np.all(V[:, 5:] == 0) and np.all(r.sigma.cpu().numpy()[5:] == 0)
    assert M.max_sine(B.numpy(), V[:, :5]) < 1e-9


def test_nonfinite_input_is_reported(ctx):
    w = C1
    X = S.generate(w).clone()
    X[17, 3] = float("nan")
    V = torch.empty(w.n, w.k, dtype=torch.float64, device="cuda")
    sig = torch.empty(w.k, dtype=torch.float64, device="cuda")
    rep = L.lspca_report()
    rc = L.lspca_fit(ctx.handle, X.cuda(), w.k, _om(w), 0, V, sig, None, None, None, rep)
    assert rc == L.ERR_NUMERIC
    assert ctx.sync_status() == L.OK  # the report consumed the status word


@pytest.mark.parametrize("dtype,where", [(torch.float32, (3, 8)), (torch.float32, (500, 1000)),
                                         (torch.bfloat16, (776, 17)), (torch.bfloat16, (0, 999))])
def test_nonfinite_reported_on_tensor_core_paths(ctx, dtype, where):
    """Gaussian Omega on FP32 / BF16 X (the tensor-core sketch, whose scan of X
    sets the FP16 scales and detects NaN/Inf): an Inf inside a 16-byte vector
    or in a row's ragged tail of a row-strided X gives ERR_NUMERIC."""
    m, n, ldx, k = 777, 1001, 1008, 16
    base = torch.randn(m, ldx, generator=torch.Generator().manual_seed(3)).to(dtype)
    base[where] = float("inf")
    X = base.cuda()[:, :n]
    V = torch.empty(n, k, dtype=torch.float32, device="cuda")
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    rep = L.lspca_report()
    rc = L.lspca_fit(ctx.handle, X, k, L.omega("gaussian", 0), 0, V, sig, None, None, None, rep)
    assert rc == L.ERR_NUMERIC
    assert ctx.sync_status() == L.OK


@pytest.mark.parametrize("bad", ["k0", "kbig", "ldx", "omega_p0", "e4m3_gauss", "null_v"])
def test_invalid_arguments(ctx, bad):
    X = torch.zeros(64, 32, dtype=torch.float32, device="cuda")
    V = torch.empty(32, 4, dtype=torch.float32, device="cuda")
    sig = torch.empty(4, dtype=torch.float64, device="cuda")
    lib = L.load()
    om = L.omega("gaussian", 0)
    args = dict(x=X.data_ptr(), xt=L.LSPCA_F32, m=64, n=32, ldx=32, k=4, om=om, v=V.data_ptr())
    if bad == "k0":
        args["k"] = 0
    elif bad == "kbig":
        args["k"] = 33
    elif bad == "ldx":
        args["ldx"] = 31
    elif bad == "omega_p0":
        args["om"] = L.omega("sparse", 0, 0)
    elif bad == "e4m3_gauss":
        args["xt"] = L.LSPCA_E4M3
    elif bad == "null_v":
        args["v"] = None
    rc = lib.lspca_fit(ctx.handle, args["x"], args["xt"], args["m"], args["n"], args["ldx"], args["k"], args["om"], 0,
                       args["v"], sig.data_ptr(), None, None, None, None)
    assert rc == L.ERR_INVALID


def test_alg4_slicing_invariance(ctx, data):
    """Algorithm 4: F summed over horizontal slices equals F of the whole (FP64 path)."""
    w, X, Xd, Om, fit = _get(data, C1)
    Xg = X.cuda()
    U = ctx.sketch(Xg, w.k, _om(w))
    F, _ = ctx.chain(Xg, U)
    parts = [0, 333, 1000, 1999, w.m]
    Fs = sum(ctx.chain(Xg[a:b], U[a:b])[0] for a, b in zip(parts[:-1], parts[1:]))
    assert torch.allclose(F, Fs, rtol=1e-12, atol=1e-12 * F.abs().max().item())


# ------------------------------------------------------------------ tensor-core projection, all X types

@pytest.mark.parametrize("dtype,k,m,n", [("f32", 20, 1000, 500), ("f32", 128, 3001, 4096), ("f32", 200, 777, 1000),
                                         ("f32", 64, 1100, 1000), ("f32", 100, 515, 2040), ("f32", 128, 1, 1000),
                                         ("f32", 64, 77, 4096),
                                         ("bf16", 64, 2049, 1024), ("bf16", 256, 513, 2048),
                                         ("bf16", 192, 1000, 1984), ("bf16", 1, 129, 512), ("bf16", 33, 1, 576),
                                         ("bf16", 128, 300, 1000),
                                         ("e4m3", 256, 1500, 4096), ("e4m3", 128, 4001, 1040),
                                         ("e4m3", 64, 700, 960), ("e4m3", 200, 257, 2112), ("e4m3", 17, 1, 64),
                                         ("e4m3", 96, 333, 1008)])
def test_project_tensor_core_paths(ctx, dtype, k, m, n):
    """Y = X V against the FP64 product of the same stored values (relative Frobenius):
    FP32 X 2e-6 (k <= 128 with n a multiple of 8: X and V in three exact BF16
    pieces each, six products, A in tensor memory; otherwise split-FP16 with
    per-row scales); BF16 X with split-BF16 V 1e-5; E4M3 X (its pitch a
    multiple of 16 bytes by the library's contract) widened exactly to FP16
    against V as an FP16 pair of 22 bits, 2e-6."""
    if dtype == "e4m3":
        w = S.WORKLOADS["e4m3_binary"].scaled(m=m, n=n, k=k)
    elif dtype == "bf16":
        w = S.WORKLOADS["bf16_dense"].scaled(m=m, n=n, k=k)
    else:
        w = S.WORKLOADS["fp32_sparse"].scaled(m=m, n=n, k=k)
    X = S.generate(w)
    g = torch.Generator().manual_seed(k * 7 + m)
    V, _ = torch.linalg.qr(torch.randn(n, k, generator=g, dtype=torch.float64))
    V32 = V.float().contiguous()  # QR returns a column-major Q; the ABI takes row-major V
    Y = ctx.project(X.cuda(), V32.cuda()).double().cpu().numpy()
    Yref = X.double().numpy() @ V32.double().numpy()
    err = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    tol = 1e-5 if dtype == "bf16" else 2e-6
    print(f"project {dtype} k={k} m={m} n={n}: rel err {err:.2e}")
    assert err < tol, err


# ------------------------------------------------------------------ BF16 and FP8 (binary) workloads

C3S = S.WORKLOADS["bf16_dense"].scaled(m=4001, n=2048)            # k = 256: two 128-row halves of F
C4S = S.WORKLOADS["e4m3_binary"].scaled(m=5001, n=1024, k=128)


def test_fit_bf16_gaussian_parity(ctx):
    """BF16 X, Gaussian Omega rounded to BF16 (the path's number format), k = 256:
    Y within 1e-4 (refined low-precision path), Procrustes-aligned."""
    w = C3S
    X = S.generate(w)
    Xd = X.double().numpy()
    Om = P.bf16_rne(P.omega_gaussian(w.omega_seed, w.n, w.k))
    fit = O.lspca_fit(Xd, Om, route="eig")
    Xg = X.cuda()
    # the sketch itself: BF16 products are exact, FP32 accumulation
    U = ctx.sketch(Xg, w.k, _om(w)).double().cpu().numpy()
    assert np.linalg.norm(U - fit["U"]) / np.linalg.norm(fit["U"]) < 1e-6
    r = ctx.fit(Xg, w.k, _om(w))
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    e = _report_errors(Y, Yref, r.V.double().cpu().numpy(), fit["V"])
    print("bf16_dense", e)
    assert e["procrustes"] < 1e-4
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-4


def test_binary_e4m3_exact_sketch_and_chain(ctx):
    """Binary X (E4M3) with the very sparse Omega: U = X Omega and F = U^T X are
    integers and come out bit-exact (FP32 holds integers below 2^24)."""
    w = C4S
    X = S.generate(w)
    Xd = X.float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    Uref = Xd @ Om
    Fref = Uref.T @ Xd
    assert np.abs(Fref).max() < 2 ** 24
    Xg = X.cuda()
    U = ctx.sketch(Xg, w.k, _om(w))
    assert np.array_equal(U.double().cpu().numpy(), Uref)
    F, _ = ctx.chain(Xg, U)
    assert np.array_equal(F.cpu().numpy(), Fref)


def test_fit_binary_e4m3_parity(ctx):
    w = C4S
    X = S.generate(w)
    Xd = X.float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    fit = O.lspca_fit(Xd, Om, route="eig")
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, _om(w))
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    e = _report_errors(Y, Yref, r.V.double().cpu().numpy(), fit["V"])
    print("e4m3_binary", e)
    assert e["procrustes"] < 1e-4


def test_fit_e4m3_not_binary_takes_the_bf16_pass_f(ctx):
    """E4M3 X with values other than 0 and 1: U is not exact in E4M3, so the
    FP8 pass F stands down, a second (gated) sketch run writes U in FP32 and
    the BF16 pass F computes F; the fit still matches the oracle."""
    w = C4S
    g = torch.Generator().manual_seed(17)
    scale = torch.rand(w.m, w.n, generator=g) * 2.75 + 0.25
    X = (S.generate(w).float() * scale).to(torch.float8_e4m3fn)
    Xd = X.float().double().numpy()
    Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p)
    Uref = Xd @ Om
    U8 = torch.from_numpy(Uref).float().to(torch.float8_e4m3fn).float().double().numpy()
    assert not np.array_equal(U8, Uref)  # the case under test: U is not exact in E4M3
    fit = O.lspca_fit(Xd, Om, route="eig")
    Xg = X.cuda()
    r = ctx.fit(Xg, w.k, _om(w))
    assert ctx.sync_status() == L.OK
    Y = ctx.project(Xg, r.V).double().cpu().numpy()
    Yref = O.project(Xd, fit["V"])
    e = _report_errors(Y, Yref, r.V.double().cpu().numpy(), fit["V"])
    print("e4m3 not binary", e)
    assert e["procrustes"] < 1e-4
    assert np.max(np.abs(r.sigma.cpu().numpy() - fit["sigma"]) / fit["sigma"]) < 1e-4

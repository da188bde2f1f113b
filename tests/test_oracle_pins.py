"""Pins of the FP64 oracle against what the paper and the mathematics fix.

CPU only.  Each test ties one oracle function to something other than
itself: published known-answer vectors, an independent library routine,
a closed form, or a proposition of the paper.  The mutation tests at the end
plant plausible mistakes in the oracle and check that a pin catches them.
"""
import os

import numpy as np
import pytest

from oracle import lspca as O
from oracle import metrics as M
from oracle import philox as P
from paper_1709_07175_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _c1():
    w = S.WORKLOADS["fp64_small"]
    X = S.generate(w).numpy()
    Om = P.omega_gaussian(w.omega_seed, w.n, w.k)
    return w, X, Om


# ---------------------------------------------------------------- Philox / Omega

def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = P.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_sparse_omega_statistics():
    """Very sparse Omega: P(-1) = P(+1) = 1/(2p), P(0) = 1 - 1/p (Sec. I-A), within 5 sigma."""
    n, k, p = 4096, 256, 64
    Om = P.omega_sparse(7, n, k, p)
    N = Om.size
    assert set(np.unique(Om)) <= {-1.0, 0.0, 1.0}
    q = 1.0 / (2 * p)
    for val in (-1.0, 1.0):
        f = np.mean(Om == val)
        assert abs(f - q) < 5 * np.sqrt(q * (1 - q) / N)
    # exact threshold: T = 2^32 / 128 for p = 64
    assert P.sparse_threshold(64) == 2 ** 25


def test_gaussian_omega_statistics():
    """Gaussian Omega entries N(0, 1) (Sec. I-A): mean, variance, kurtosis within 5 sigma."""
    Om = P.omega_gaussian(3, 4096, 128)
    x = Om.ravel()
    N = x.size
    assert abs(x.mean()) < 5 / np.sqrt(N)
    assert abs(x.var() - 1) < 5 * np.sqrt(2.0 / N)
    kurt = np.mean(x ** 4) / x.var() ** 2
    assert abs(kurt - 3) < 5 * np.sqrt(24.0 / N)
    # values are FP32-representable
    assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    # independent columns: sample correlation of two columns is O(1/sqrt(n))
    c = np.corrcoef(Om[:, 0], Om[:, 1])[0, 1]
    assert abs(c) < 5 / np.sqrt(4096)


def test_omega_seed_and_layout():
    """Different seeds / tags give different streams; entry (i, j) only depends on (seed, i, j)."""
    a = P.omega_gaussian(0, 64, 12)
    b = P.omega_gaussian(1, 64, 12)
    assert not np.array_equal(a, b)
    # the leading block of a larger matrix equals the smaller matrix
    big = P.omega_gaussian(0, 128, 20)
    assert np.array_equal(big[:64, :12], a)
    sp = P.omega_sparse(5, 128, 20, 4)
    assert np.array_equal(P.omega_sparse(5, 64, 12, 4), sp[:64, :12])


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(0).standard_normal(10000) * 10
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(P.bf16_rne(x), ref)


# ---------------------------------------------------------------- decompositions

@pytest.mark.parametrize("k,n", [(5, 9), (8, 40), (20, 500)])
def test_onesided_jacobi_matches_library_svd(k, n):
    rng = np.random.default_rng(k * 100 + n)
    F = rng.standard_normal((k, n)) * np.logspace(0, -3, k)[:, None]
    V, s, _ = O.svd_onesided_jacobi(F)
    s_ref = np.linalg.svd(F, compute_uv=False)
    assert np.allclose(s, s_ref, rtol=1e-12, atol=0)
    _, _, vt = np.linalg.svd(F, full_matrices=False)
    assert M.max_sine(vt.T, V) < 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-13
    # F = (F V) V^T
    assert np.linalg.norm(F - (F @ V) @ V.T) < 1e-13 * np.linalg.norm(F)
    # columns are individual singular vectors: F^T F v_i = s_i^2 v_i
    R = F.T @ (F @ V) - V * s ** 2
    assert np.abs(R).max() < 1e-12 * s[0] ** 2


@pytest.mark.parametrize("k", [3, 8, 21, 64])
def test_eig_jacobi_matches_library_eigh(k):
    rng = np.random.default_rng(k)
    A = rng.standard_normal((k, 3 * k))
    H = A @ A.T
    lam, W, _ = O.eig_jacobi(H)
    lam_ref = np.linalg.eigh(H)[0][::-1]
    assert np.allclose(lam, lam_ref, rtol=0, atol=1e-12 * lam_ref[0])
    assert np.abs(W.T @ W - np.eye(k)).max() < 1e-13
    assert np.abs(H @ W - W * lam).max() < 1e-12 * lam[0]


def test_eig_route_equals_svd_route():
    """Table footnote: eig(F F^T) with D = Lambda^1/2, V = F^T W D^-1 is the truncated SVD."""
    w, X, Om = _c1()
    F = O.chain(O.sketch(X, Om), X)
    Ve, se, re = O.decompose_eig(F, w.m, w.n)
    Vs, ss, rs = O.decompose_svd(F, w.m, w.n)
    assert re == rs == w.k
    assert np.allclose(se, ss, rtol=1e-10)
    assert M.max_sine(Vs, Ve) < 1e-10
    # per-column agreement after the sign rule (c1 has distinct singular values)
    gaps = np.min(np.abs(np.diff(ss))) / ss[0]
    assert gaps > 1e-6
    assert np.abs(Ve - Vs).max() < 1e-8


def test_householder_qr_matches_library():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((300, 17))
    Q, R = O.householder_qr(A)
    assert np.abs(Q @ R - A).max() < 1e-13 * np.abs(A).max() * 10
    assert np.abs(Q.T @ Q - np.eye(17)).max() < 1e-13
    assert np.allclose(np.tril(R, -1), 0)
    _, Rl = np.linalg.qr(A)
    assert np.allclose(np.abs(R), np.abs(Rl), rtol=1e-11, atol=1e-13)


def test_sign_rule_and_ties():
    V = np.array([[0.6, -0.8, 0.5], [-0.8, 0.6, -0.5]])
    out = O.sign_rule(V)
    assert np.array_equal(out[:, 0], [-0.6, 0.8])
    assert np.array_equal(out[:, 1], [0.8, -0.6])
    # tie |0.5| = |-0.5|: the lowest index decides
    assert np.array_equal(out[:, 2], [0.5, -0.5])


# ---------------------------------------------------------------- propositions

def test_prop1_lazy_amd_equals_amd():
    """Prop. 1: Q Q^T X = U' U^T X with U' = U (U^T U)^-1."""
    w, X, Om = _c1()
    U = O.sketch(X, Om)
    Q, _ = O.householder_qr(U)
    G = O.gram(U)
    lazy = U @ np.linalg.solve(G, U.T @ X)
    amd = Q @ (Q.T @ X)
    assert np.linalg.norm(lazy - amd) / np.linalg.norm(X) < 1e-12


def test_prop2_equal_spans():
    """Prop. 2: V^s and V^l span the same subspace (max principal-angle sine <= 1e-10)."""
    w, X, Om = _c1()
    lz = O.lspca_fit(X, Om, route="svd")
    sp = O.spca_fit(X, Om, route="svd")
    assert M.max_sine(sp["V"], lz["V"]) < 1e-10
    assert M.chordal(sp["V"], lz["V"]) < 1e-10
    # both bases are orthonormal; the footnote of Sec. III-B.2 says V^T = V^T V V^T
    for V in (sp["V"], lz["V"]):
        assert np.abs(V.T @ V - np.eye(w.k)).max() < 1e-13
    # the spans are span(X^T u_1, ..., X^T u_l)
    XtU = X.T @ lz["U"]
    Qx, _ = np.linalg.qr(XtU)
    assert M.max_sine(Qx, lz["V"]) < 1e-10


def test_prop3_equal_pairwise_distances():
    """Prop. 3: d(pi^s x_i, pi^s x_j) = d(pi^l x_i, pi^l x_j) <= d(x_i, x_j)."""
    w, X, Om = _c1()
    Vl = O.lspca_fit(X, Om, route="svd")["V"]
    Vs = O.spca_fit(X, Om, route="svd")["V"]
    Yl, Ys = O.project(X, Vl), O.project(X, Vs)
    rng = np.random.default_rng(11)
    i = rng.integers(0, w.m, 10000)
    j = rng.integers(0, w.m, 10000)
    keep = i != j
    i, j = i[keep], j[keep]
    dl = np.linalg.norm(Yl[i] - Yl[j], axis=1)
    ds = np.linalg.norm(Ys[i] - Ys[j], axis=1)
    dx = np.linalg.norm(X[i] - X[j], axis=1)
    assert np.max(np.abs(ds - dl) / dl) < 1e-10
    assert np.all(dl <= dx * (1 + 1e-12))
    # equivalently W = V^sT V^l is orthogonal and Y^l = Y^s W
    W = Vs.T @ Vl
    assert np.abs(W.T @ W - np.eye(w.k)).max() < 1e-12
    assert np.linalg.norm(Ys @ W - Yl) / np.linalg.norm(Yl) < 1e-10


def test_rank_r_recovery():
    """Exactly rank-r X (r <= k): both fits recover range(B), the brute-force
    top-r right singular space, and report rank r."""
    X, B = (t.numpy() for t in S.rank_r_exact(60, 40, 5, seed=3))
    Om = P.omega_gaussian(9, 40, 8)
    lz = O.lspca_fit(X, Om, route="eig")
    lz_svd = O.lspca_fit(X, Om, route="svd")
    sp = O.spca_fit(X, Om, route="svd")
    _, _, vt = np.linalg.svd(X)
    top = vt[:5].T
    for fit in (lz, lz_svd, sp):
        assert fit["rank"] == 5
        assert np.count_nonzero(fit["sigma"]) == 5
        assert M.max_sine(top, fit["V"][:, :5]) < 1e-10
        assert M.max_sine(B, fit["V"][:, :5]) < 1e-10
        assert np.all(fit["V"][:, 5:] == 0)


def _lazy_residual_norm(X, U):
    """||X - U' U^T X||_2 with U' = U (U^T U)^-1 (Lemma 1), by library routines."""
    R = X - U @ np.linalg.solve(U.T @ U, U.T @ X)
    return np.linalg.norm(R, 2)


def test_oversampled_corollary_bound():
    """Corollary of Sec. II (Gaussian Omega, l >= k + 2): the mean over draws of
    ||X - U' U^T X||_2 is at most [1 + 4 sqrt(l) / (l - k - 1) sqrt(min(m, n))]
    sigma_{k+1}; and no draw beats sigma_{l+1}, the best rank-l error."""
    rng = np.random.default_rng(21)
    m, n, k, l = 300, 120, 6, 12
    A, _ = np.linalg.qr(rng.standard_normal((m, 40)))
    B, _ = np.linalg.qr(rng.standard_normal((n, 40)))
    X = A @ np.diag(0.8 ** np.arange(40)) @ B.T + 1e-3 * rng.standard_normal((m, n))
    sv = np.linalg.svd(X, compute_uv=False)
    errs = []
    for seed in range(8):
        U = O.sketch(X, P.omega_gaussian(seed, n, l))
        e = _lazy_residual_norm(X, U)
        assert e >= sv[l] * (1 - 1e-10)
        errs.append(e)
    bound = (1 + 4 * np.sqrt(l) / (l - k - 1) * np.sqrt(min(m, n))) * sv[k]
    assert np.mean(errs) <= bound
    # oversampling helps: the mean error with l = k + 6 is below the one with l = k
    errs_k = [_lazy_residual_norm(X, O.sketch(X, P.omega_gaussian(seed, n, k))) for seed in range(8)]
    assert np.mean(errs) < np.mean(errs_k)


def test_oversampled_fit_is_the_top_k_of_the_l_column_fit():
    """l > k: V and sigma are the top k singular triplets of F = U^T X for the
    l-column Omega (library SVD of F); the full l-dimensional spans of Lazy and
    SPCA agree (Prop. 2 at l), while their top-k truncations differ in general;
    with l = n, SPCA's top k is the data's own top-k right singular space."""
    rng = np.random.default_rng(22)
    m, n, k, l = 200, 40, 5, 9
    X = rng.standard_normal((m, n)) @ np.diag(0.9 ** np.arange(n))
    Om = P.omega_gaussian(3, n, l)
    lz = O.lspca_fit_oversampled(X, Om, k)
    assert lz["V"].shape == (n, k) and lz["sigma"].shape == (k,) and lz["rank"] == k
    F = O.sketch(X, Om).T @ X
    _, s_ref, vt = np.linalg.svd(F, full_matrices=False)
    assert np.max(np.abs(lz["sigma"] - s_ref[:k]) / s_ref[:k]) < 1e-10
    assert M.max_sine(vt[:k].T, lz["V"]) < 1e-9
    sp = O.spca_fit(X, Om, route="svd")
    assert M.max_sine(lz["full"]["V"], sp["V"]) < 1e-10
    assert M.max_sine(lz["V"], sp["V"][:, :k]) > 1e-6
    # l = n: span(U) = range(X); Q^T X has X's singular values
    spn = O.spca_fit(X, P.omega_gaussian(4, n, n), route="svd")
    _, s_x, vt_x = np.linalg.svd(X, full_matrices=False)
    assert M.max_sine(vt_x[:k].T, spn["V"][:, :k]) < 1e-8
    assert np.max(np.abs(spn["sigma"][:k] - s_x[:k]) / s_x[:k]) < 1e-10


def test_oversampled_rank_r_recovery():
    """Exactly rank-r X with r < k < l: rank r, and V's first r columns span range(B)."""
    X, B = (t.numpy() for t in S.rank_r_exact(60, 40, 4, seed=5))
    fit = O.lspca_fit_oversampled(X, P.omega_gaussian(11, 40, 10), 6)
    assert fit["rank"] == 4
    assert M.max_sine(B, fit["V"][:, :4]) < 1e-10
    assert np.all(fit["V"][:, 4:] == 0) and np.all(fit["sigma"][4:] == 0)


def test_closed_form_selector_omega():
    """Omega = [e_1 ... e_k]: U = X[:, :k] and F = X[:, :k]^T X."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50, 12))
    Om = np.eye(12)[:, :4]
    U = O.sketch(X, Om)
    assert np.array_equal(U, X[:, :4])
    F = O.chain(U, X)
    assert np.allclose(F, X[:, :4].T @ X, rtol=0, atol=1e-13)
    assert np.allclose(F[:, :4], F[:, :4].T)


def test_closed_form_identity_data():
    """X = I_n: F = Omega^T and V^l spans range(Omega)."""
    n, k = 30, 6
    Om = P.omega_gaussian(4, n, k)
    X = np.eye(n)
    F = O.chain(O.sketch(X, Om), X)
    assert np.array_equal(F, Om.T)
    V = O.lspca_fit(X, Om, route="eig")["V"]
    Qo, _ = np.linalg.qr(Om)
    assert M.max_sine(Qo, V) < 1e-12


def test_alg2_equals_alg4_any_slicing():
    """Algorithm 4 (slices) gives Algorithm 2's F and G up to summation order."""
    w, X, Om = _c1()
    U = O.sketch(X, Om)
    F2, G2 = O.chain(U, X), O.gram(U)
    for bounds in ([0, w.m], [0, 1, 777, 1500, w.m], list(range(0, w.m, 128)) + [w.m]):
        F4, G4 = O.streaming_lazy(X, Om, bounds)
        assert np.abs(F4 - F2).max() < 1e-13 * np.abs(F2).max()
        assert np.abs(G4 - G2).max() < 1e-13 * np.abs(G2).max()


def test_alg3_streaming_spca_equals_alg1():
    """Algorithm 3: R^-T U^T X = Q^T X (rows up to the signs of R's diagonal)."""
    w, X, Om = _c1()
    U = O.sketch(X, Om)
    Q, R1 = O.householder_qr(U)
    ref = Q.T @ X
    st = O.streaming_spca(X, Om, [0, 300, 1000, 1999, w.m])
    d = np.sign(np.diag(st["R"])) * np.sign(np.diag(R1))
    assert np.linalg.norm(st["F"] * d[:, None] - ref) / np.linalg.norm(ref) < 1e-12
    # R^T R = U^T U (the Gram of the sketch)
    G = O.gram(U)
    assert np.abs(st["R"].T @ st["R"] - G).max() < 1e-12 * np.abs(G).max()


def test_chordal_distance_definition():
    """metrics.chordal equals ||A A^T - B B^T||_F (Experiment 2's definition)."""
    rng = np.random.default_rng(2)
    A, _ = np.linalg.qr(rng.standard_normal((40, 5)))
    B, _ = np.linalg.qr(rng.standard_normal((40, 5)))
    direct = np.linalg.norm(A @ A.T - B @ B.T)
    assert abs(M.chordal(A, B) - direct) < 1e-12
    assert M.chordal(A, A) < 1e-14
    assert M.max_sine(A, A @ np.linalg.qr(rng.standard_normal((5, 5)))[0]) < 1e-14


def test_procrustes_recovers_rotation():
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((200, 6))
    W, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    assert M.procrustes_rel(Y @ W, Y) < 1e-14
    assert M.signaligned_rel(-Y, Y) == 0.0


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible oracle mistakes on the CPU and check that a pin fails."""
    w, X, Om = _c1()
    # (a) eigen rotation with the wrong sign of s: Jacobi no longer diagonalises
    orig = O.eig_jacobi

    def bad_eig(H, tol=1e-15, max_sweeps=3):
        lam, W, s = orig(H, tol, max_sweeps=1)
        return lam, W[:, ::-1] if W.shape[1] > 1 else W, s
    monkeypatch.setattr(O, "eig_jacobi", bad_eig)
    F = O.chain(O.sketch(X, Om), X)
    Ve, _, _ = O.decompose_eig(F, w.m, w.n)
    Vs, _, _ = O.decompose_svd(F, w.m, w.n)
    assert np.abs(Ve - Vs).max() > 1e-3
    monkeypatch.setattr(O, "eig_jacobi", orig)
    # (b) transposed data in the chain (F from X^T X instead of U^T X) breaks Prop. 2
    U = O.sketch(X, Om)
    F_bad = (X.T @ X)[: w.k]
    Vb, _, _ = O.decompose_svd(F_bad, w.m, w.n)
    Vg, _, _ = O.decompose_svd(O.chain(U, X), w.m, w.n)
    assert M.max_sine(Vg, Vb) > 1e-3
    # (c) a dropped slice in Algorithm 4 breaks the Alg 2 = Alg 4 pin
    F4, _ = O.streaming_lazy(X[:1500], Om, [0, 1500])
    assert np.abs(F4 - O.chain(U, X)).max() > 1e-6
    # (d) an oversampled fit that keeps the last k triplets instead of the top k
    # fails the top-k pin (sigma against the library SVD of F)
    rng = np.random.default_rng(22)
    Xo = rng.standard_normal((200, 40)) @ np.diag(0.9 ** np.arange(40))
    Omo = P.omega_gaussian(3, 40, 9)
    full = O.lspca_fit(Xo, Omo)
    s_ref = np.linalg.svd(O.sketch(Xo, Omo).T @ Xo, compute_uv=False)
    assert np.max(np.abs(full["sigma"][-5:] - s_ref[:5]) / s_ref[:5]) > 1e-3


def test_sparse_oracle_equals_dense_oracle():
    """The sparse-input oracle (scipy sparse products) is the dense oracle on the
    densified matrix: F to 1e-13, V and sigma to 1e-10.  The CSR generator's
    output is valid CSR (offsets, sorted distinct columns per row)."""
    sp = pytest.importorskip("scipy.sparse")
    rp, c, v = S.sparse_csr(400, 300, 0.02, seed=1)
    rp, c, v = rp.numpy(), c.numpy(), v.numpy()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == c.size == v.size
    for i in range(400):
        cols = c[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0) and (cols.size == 0 or (cols[0] >= 0 and cols[-1] < 300))
    Xs = sp.csr_matrix((v, c, rp), shape=(400, 300))
    Om = P.omega_gaussian(2, 300, 16)
    a = O.lspca_fit_sparse(Xs, Om)
    b = O.lspca_fit(Xs.toarray(), Om)
    assert np.max(np.abs(a["F"] - b["F"])) <= 1e-13 * np.max(np.abs(b["F"]))
    assert np.max(np.abs(a["sigma"] - b["sigma"]) / b["sigma"]) < 1e-10
    assert M.max_sine(a["V"], b["V"]) < 1e-10

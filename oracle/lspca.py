"""FP64 oracle of Lazy SPCA and SPCA (Wojnowicz et al., arXiv 1709.07175).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here is plain FP64 numpy.  A matrix product (``@``) is the only
library primitive used on the method's path; the SVD, the symmetric
eigensolver and the Householder QR are written out so that independent
library routines can pin them in the tests.

Notation follows the paper: X is m x n with samples as rows (Sec. I-A), Omega
is n x l with l = k (no oversampling, as in Experiment 1; lspca_fit_oversampled
takes l > k and keeps the top k), U = X Omega is m x l, F = U^T X is l x n,
V is n x k, the reduction is Y = X V (m x k).
X is never centred (Sec. I-B, "uncentered" PCA).

Readings where the paper is silent (shared with the GPU library):
* scale c of Eq. 1 is 1 (V does not depend on it; sigma scales by 1/c);
* order: descending singular values;
* sign: each column of V is flipped so its largest-magnitude entry is
  positive, ties to the lowest index (the footnote of Sec. III-B.2 notes the
  bases are not unique);
* rank: the eigen route (table footnote) drops eigenvalues
  lambda_i <= max(m, n) 2^-52 lambda_1; the SVD route drops
  sigma_i <= max(m, n) 2^-52 sigma_1; dropped columns of V and their sigma
  are set to zero and the rank is reported (the paper defers rank-deficient U
  to future work, footnote of Corollary 1).
"""
from __future__ import annotations

import numpy as np

EPS64 = 2.0 ** -52


# ----------------------------------------------------------------------------
# Eq. 1 and Algorithms 2 / 4: the sketch and the projection chain
# ----------------------------------------------------------------------------

def sketch(X: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """U = X Omega (Eq. 1 with c = 1; Algorithm 2 step 1)."""
    return np.asarray(X, np.float64) @ np.asarray(Omega, np.float64)


def chain(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """F = U^T X (Algorithm 2 step 2)."""
    return np.asarray(U, np.float64).T @ np.asarray(X, np.float64)


def gram(U: np.ndarray) -> np.ndarray:
    """G = U^T U, the k x k Gram of the sketch (U' = U G^-1, Lemma 1)."""
    U = np.asarray(U, np.float64)
    return U.T @ U


def streaming_lazy(X: np.ndarray, Omega: np.ndarray, bounds) -> tuple:
    """Algorithm 4: F = sum over horizontal slices X_s of (X_s Omega)^T X_s.

    ``bounds`` are the slice edges [0, b1, ..., m].  Returns (F, G) where G
    sums U_s^T U_s over the same slices.
    """
    X = np.asarray(X, np.float64)
    k = Omega.shape[1]
    F = np.zeros((k, X.shape[1]))
    G = np.zeros((k, k))
    for a, b in zip(bounds[:-1], bounds[1:]):
        Us = sketch(X[a:b], Omega)
        F += chain(Us, X[a:b])
        G += gram(Us)
    return F, G


# ----------------------------------------------------------------------------
# Truncated SVD of the small factor F (Algorithms 1-4, last step)
# ----------------------------------------------------------------------------

def _round_robin(k: int):
    """Pairings of a round-robin tournament: k-1 (or k) rounds of disjoint pairs."""
    players = list(range(k)) + ([-1] if k % 2 else [])
    r = len(players)
    rounds = []
    for _ in range(r - 1):
        pairs = [(players[i], players[r - 1 - i]) for i in range(r // 2)]
        rounds.append([(min(p, q), max(p, q)) for p, q in pairs if p >= 0 and q >= 0])
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def svd_onesided_jacobi(F: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Truncated SVD of F (k x n) by one-sided (Hestenes) Jacobi on F^T.

    Plane rotations J are applied from the right to A = F^T until all column
    pairs are orthogonal (|a_p . a_q| <= tol ||a_p|| ||a_q||).  Then
    F^T J = V Sigma: the singular values are the column norms and V holds the
    normalised columns.  Returns (V n x k, sigma descending, sweeps).
    """
    A = np.array(F, dtype=np.float64).T.copy()
    n, k = A.shape
    rounds = _round_robin(k)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for pairs in rounds:
            if not pairs:
                continue
            p = np.array([a for a, _ in pairs])
            q = np.array([b for _, b in pairs])
            ap, aq = A[:, p], A[:, q]
            alpha = np.einsum("ij,ij->j", ap, ap)
            beta = np.einsum("ij,ij->j", aq, aq)
            gamma = np.einsum("ij,ij->j", ap, aq)
            act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            if not act.any():
                continue
            rotated = True
            g = np.where(act, gamma, 1.0)
            zeta = (beta - alpha) / (2.0 * g)
            t = np.sign(zeta) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            t = np.where(zeta == 0.0, 1.0, t)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            c = np.where(act, c, 1.0)
            s = np.where(act, s, 0.0)
            A[:, p] = c * ap - s * aq
            A[:, q] = s * ap + c * aq
        if not rotated:
            break
    sigma = np.sqrt(np.einsum("ij,ij->j", A, A))
    order = np.argsort(-sigma, kind="stable")
    sigma = sigma[order]
    A = A[:, order]
    V = np.zeros_like(A)
    nz = sigma > 0
    V[:, nz] = A[:, nz] / sigma[nz]
    return V, sigma, sweeps


def eig_jacobi(H: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Symmetric eigendecomposition H = W Lambda W^T by two-sided Jacobi.

    Each rotation zeroes H_pq (|H_pq| > tol sqrt(|H_pp H_qq|)); rotations of a
    round act on disjoint index pairs.  Returns (lambda descending, W, sweeps).
    """
    A = np.array(H, dtype=np.float64)
    k = A.shape[0]
    W = np.eye(k)
    rounds = _round_robin(k)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for pairs in rounds:
            if not pairs:
                continue
            p = np.array([a for a, _ in pairs])
            q = np.array([b for _, b in pairs])
            apq = A[p, q]
            app = A[p, p]
            aqq = A[q, q]
            act = np.abs(apq) > tol * np.sqrt(np.abs(app * aqq))
            if not act.any():
                continue
            rotated = True
            g = np.where(act, apq, 1.0)
            tau = (aqq - app) / (2.0 * g)
            t = np.sign(tau) / (np.abs(tau) + np.sqrt(1.0 + tau * tau))
            t = np.where(tau == 0.0, 1.0, t)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = t * c
            c = np.where(act, c, 1.0)
            s = np.where(act, s, 0.0)
            # A <- J^T A J with J the product of the disjoint rotations
            rp, rq = A[p, :].copy(), A[q, :].copy()
            A[p, :] = c[:, None] * rp - s[:, None] * rq
            A[q, :] = s[:, None] * rp + c[:, None] * rq
            cp, cq = A[:, p].copy(), A[:, q].copy()
            A[:, p] = c * cp - s * cq
            A[:, q] = s * cp + c * cq
            wp, wq = W[:, p].copy(), W[:, q].copy()
            W[:, p] = c * wp - s * wq
            W[:, q] = s * wp + c * wq
        if not rotated:
            break
    lam = np.diag(A).copy()
    order = np.argsort(-lam, kind="stable")
    return lam[order], W[:, order], sweeps


def sign_rule(V: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-|.| entry is positive (lowest index on ties)."""
    V = np.array(V, dtype=np.float64)
    idx = np.argmax(np.abs(V), axis=0)  # argmax returns the first maximum
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1.0
    return V * s


def decompose_svd(F: np.ndarray, m: int, n: int):
    """Reference route: truncated SVD of F, rank rule on sigma.

    Returns (V, sigma, rank) after the sign and rank rules.
    """
    V, sigma, _ = svd_onesided_jacobi(F)
    tol = max(m, n) * EPS64 * (sigma[0] if sigma.size else 0.0)
    keep = sigma > tol
    V = sign_rule(V)
    V[:, ~keep] = 0.0
    sigma = np.where(keep, sigma, 0.0)
    return V, sigma, int(keep.sum())


def decompose_eig(F: np.ndarray, m: int, n: int):
    """Paper route (table footnote): F F^T = W Lambda W^T, D = Lambda^1/2,
    V = F^T W D^-1.  Rank rule on lambda.  Returns (V, sigma, rank)."""
    F = np.asarray(F, np.float64)
    H = F @ F.T
    lam, W, _ = eig_jacobi(H)
    tol = max(m, n) * EPS64 * (lam[0] if lam.size else 0.0)
    keep = lam > tol
    sigma = np.where(keep, np.sqrt(np.where(keep, lam, 1.0)), 0.0)
    V = np.zeros((F.shape[1], F.shape[0]))
    V[:, keep] = (F.T @ W[:, keep]) / sigma[keep]
    V = sign_rule(V)
    V[:, ~keep] = 0.0
    return V, sigma, int(keep.sum())


# ----------------------------------------------------------------------------
# Householder QR (Algorithms 1 and 3)
# ----------------------------------------------------------------------------

def householder_qr(A: np.ndarray):
    """Thin QR of A (m x k, m >= k) by Householder reflections, Q formed explicitly.

    Column j: v = a_j(j:) + sign(a_jj) ||a_j(j:)|| e_1, H_j = I - 2 v v^T / v^T v.
    Returns (Q m x k with orthonormal columns, R k x k upper triangular).
    """
    R = np.array(A, dtype=np.float64)
    m, k = R.shape
    vs = []
    for j in range(k):
        x = R[j:, j]
        nx = np.sqrt(x @ x)
        v = x.copy()
        v[0] += (1.0 if x[0] >= 0 else -1.0) * nx
        vv = v @ v
        if vv > 0:
            R[j:, j:] -= np.outer(v, (2.0 / vv) * (v @ R[j:, j:]))
        vs.append((v, vv))
    Q = np.zeros((m, k))
    Q[:k, :k] = np.eye(k)
    for j in range(k - 1, -1, -1):
        v, vv = vs[j]
        if vv > 0:
            Q[j:, :] -= np.outer(v, (2.0 / vv) * (v @ Q[j:, :]))
    return Q, np.triu(R[:k, :k])


# ----------------------------------------------------------------------------
# The fits (Algorithms 1-4) and the reduction maps (Sec. III-B.2)
# ----------------------------------------------------------------------------

def lspca_fit(X: np.ndarray, Omega: np.ndarray, route: str = "eig") -> dict:
    """Lazy SPCA, Algorithm 2: U = X Omega; F = U^T X; truncated SVD of F.

    ``route`` selects the decomposition: "eig" (table footnote, the GPU's
    route) or "svd" (one-sided Jacobi).  Returns V^l, sigma~, rank, U, F, G.
    """
    X = np.asarray(X, np.float64)
    m, n = X.shape
    U = sketch(X, Omega)
    F = chain(U, X)
    dec = decompose_eig if route == "eig" else decompose_svd
    V, sigma, rank = dec(F, m, n)
    return {"V": V, "sigma": sigma, "rank": rank, "U": U, "F": F, "G": gram(U)}


def lspca_fit_sparse(Xs, Omega: np.ndarray, route: str = "eig") -> dict:
    """Lazy SPCA (Algorithm 2) of a sparse X (a scipy.sparse matrix, rows =
    samples): U = X Omega and F = U^T X by sparse-dense matrix products in
    FP64, whose cost is proportional to nnz(X) (Prop. 4); then the same
    truncated SVD of F.  Returns V^l, sigma~, rank, U, F."""
    m, n = Xs.shape
    Xs = Xs.astype(np.float64)
    U = np.asarray(Xs @ np.asarray(Omega, np.float64))
    F = np.asarray((Xs.T @ U).T)
    dec = decompose_eig if route == "eig" else decompose_svd
    V, sigma, rank = dec(F, m, n)
    return {"V": V, "sigma": sigma, "rank": rank, "U": U, "F": F}


def lspca_fit_oversampled(X: np.ndarray, Omega: np.ndarray, k: int, route: str = "eig") -> dict:
    """Lazy SPCA with oversampling (Sec. I-B: l = k + p columns of Omega, a
    small oversampling parameter p): the fit of Algorithm 2 with the n x l
    Omega, then the truncated SVD of F = U^T X kept to its top k singular
    triplets (V's first k columns, sigma's first k values; rank capped at k).
    Returns V (n x k), sigma (k), rank and the l-column fit under "full"."""
    full = lspca_fit(X, Omega, route)
    return {"V": full["V"][:, :k], "sigma": full["sigma"][:k], "rank": min(full["rank"], k), "full": full}


def spca_fit(X: np.ndarray, Omega: np.ndarray, route: str = "svd") -> dict:
    """SPCA, Algorithm 1: U = X Omega; Q, R = qr(U); F = Q^T X; SVD of F."""
    X = np.asarray(X, np.float64)
    m, n = X.shape
    U = sketch(X, Omega)
    Q, R = householder_qr(U)
    Fs = Q.T @ X
    dec = decompose_eig if route == "eig" else decompose_svd
    V, sigma, rank = dec(Fs, m, n)
    return {"V": V, "sigma": sigma, "rank": rank, "U": U, "Q": Q, "R": R, "F": Fs}


def streaming_spca(X: np.ndarray, Omega: np.ndarray, bounds) -> dict:
    """Algorithm 3: per slice F += U_s^T X_s and R <- qr([R; U_s]).R; then
    F <- R^-T F.  Returns F_s = R^-T U^T X and the final R."""
    X = np.asarray(X, np.float64)
    k = Omega.shape[1]
    F = np.zeros((k, X.shape[1]))
    R = None
    for a, b in zip(bounds[:-1], bounds[1:]):
        Us = sketch(X[a:b], Omega)
        F += chain(Us, X[a:b])
        stack = Us if R is None else np.vstack([R, Us])
        _, R = householder_qr(stack)
    # F <- R^-T F by forward substitution on R^T (lower triangular)
    L = R.T
    Fs = np.zeros_like(F)
    for i in range(k):
        Fs[i] = (F[i] - L[i, :i] @ Fs[:i]) / L[i, i]
    return {"F": Fs, "R": R}


def project(X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Reduction map pi(x) = V^T x applied to every row: Y = X V (Sec. III-B.2)."""
    return np.asarray(X, np.float64) @ np.asarray(V, np.float64)

"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data; it holds none of the method's arithmetic, so the
GPU library and the FP64 oracle can both consume its output.  The paper's two
datasets (the malware corpus of Experiment 1 and the Home Depot TF-IDF set of
Experiment 2) are not available; these generators stand in for them.

Workloads (the sigma index i runs 1..r):

* ``fp64_small``   2,000 x 500, X = A diag(10 * 0.85^i) B^T + N(0, 0.01^2),
                   r = 30, FP64, k = 20, Gaussian Omega.
* ``fp32_sparse``  200,000 x 4,096, sigma_i = 1/i over r = 512,
                   noise N(0, 1e-3^2), FP32, k = 128, very sparse Omega p = 64.
* ``bf16_dense``   1,000,000 x 8,192, sigma_i = exp(-i/200) over r = 1,024,
                   noise N(0, 1e-3^2), stored BF16, k = 256, Gaussian Omega.
* ``e4m3_binary``  4,600,000 x 4,096 binary features, column rates
                   p_j ~ Beta(0.5, 9.5) (5 % mean density), stored FP8 E4M3,
                   k = 256, very sparse Omega p = 64.
* ``sparse_tfidf`` (``sparse_csr``) 74,067 x 28,606 CSR at density 0.000513,
                   the shape of Experiment 2's TF-IDF matrix: per-row counts
                   Poisson(density n), columns drawn with Zipf-like weights
                   (j + 10)^-0.9 (a few frequent terms, a long tail), values
                   0.5 + |N(0, 1)| in FP32; k = 128, very sparse Omega with
                   p = round(sqrt(n)) = 169.

A and B are orthonormal (reduced QR of Gaussian draws, on the CPU in FP64 for
every target device, except the left factor of more than 250,000 rows on a
CUDA device: drawn and QR-factored there in FP32).  Rows of the noise are drawn in fixed chunks from
per-chunk generators on the target device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    k: int
    dtype: str           # storage / arithmetic type of X: "f64", "f32", "bf16", "e4m3"
    omega: str           # "gaussian" or "sparse"
    p: int = 0           # very sparse parameter (Sec. I-A)
    r: int = 0
    noise: float = 0.0
    spectrum: str = ""
    data_seed: int = 1
    omega_seed: int = 0
    extra: dict = field(default_factory=dict)

    def sigmas(self) -> np.ndarray:
        i = np.arange(1, self.r + 1, dtype=np.float64)
        if self.spectrum == "geom0.85":
            return 10.0 * 0.85 ** i
        if self.spectrum == "powerlaw1":
            return 1.0 / i
        if self.spectrum == "exp200":
            return np.exp(-i / 200.0)
        if self.spectrum == "pow2":  # steep decay, sigma_i = 2^-i
            return 2.0 ** -i
        raise ValueError(self.spectrum)

    def scaled(self, m: int | None = None, n: int | None = None, k: int | None = None) -> "Workload":
        """Same generator recipe at other sizes (rank clipped to min(m, n))."""
        mm = self.m if m is None else m
        nn = self.n if n is None else n
        kk = self.k if k is None else k
        r = min(self.r, mm, nn) if self.r else 0
        return Workload(self.name, mm, nn, kk, self.dtype, self.omega, self.p, r, self.noise,
                        self.spectrum, self.data_seed, self.omega_seed, dict(self.extra))


# A steep spectrum (sigma_i = 2^-i over rank 60, noise N(0, 1e-12^2)), FP64:
# the eigenvalues of F F^T then span many decades, which exercises the graded
# k x k eigensolve (no paper workload; a stress case for the eigen route).
STEEP = Workload("steep_pow2", 3000, 1000, 64, "f64", "gaussian", 0, 60, 1e-12, "pow2", 7, 0)


WORKLOADS = {
    "fp64_small": Workload("fp64_small", 2000, 500, 20, "f64", "gaussian", 0, 30, 0.01, "geom0.85", 1, 0),
    "fp32_sparse": Workload("fp32_sparse", 200_000, 4096, 128, "f32", "sparse", 64, 512, 1e-3, "powerlaw1", 2, 0),
    "bf16_dense": Workload("bf16_dense", 1_000_000, 8192, 256, "bf16", "gaussian", 0, 1024, 1e-3, "exp200", 3, 0),
    "e4m3_binary": Workload("e4m3_binary", 4_600_000, 4096, 256, "e4m3", "sparse", 64, 0, 0.0, "", 4, 0,
                            {"beta_a": 0.5, "beta_b": 9.5}),
}

TORCH_DTYPES = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
                "e4m3": torch.float8_e4m3fn}


def _orthonormal(rows: int, r: int, gen: torch.Generator) -> torch.Tensor:
    """Orthonormal rows x r factor: reduced QR of a Gaussian draw (CPU, FP64)."""
    g = torch.randn(rows, r, generator=gen, dtype=torch.float64)
    q, _ = torch.linalg.qr(g, mode="reduced")
    return q


# Above this many rows, a CUDA target draws the left factor A on the device.
DEVICE_FACTOR_ROWS = 250_000


def lowrank_plus_noise(w: Workload, device="cpu", chunk_rows: int = 65536,
                       out: torch.Tensor | None = None) -> torch.Tensor:
    """X = A diag(sigma) B^T + noise, rounded once to the storage dtype.

    The orthonormal factors A and B always come from the CPU generator in FP64
    (so every device sees the same factors); the noise is drawn on ``device``
    (FP64 on the CPU, FP32 on a GPU) from per-chunk generators.  Returns an
    (m, n) row-major tensor on ``device`` in ``TORCH_DTYPES[w.dtype]``.
    """
    dev = torch.device(device)
    work = torch.float64 if dev.type == "cpu" else torch.float32
    gen = torch.Generator()
    gen.manual_seed(int(w.data_seed) * 1_000_003 + 17)
    if dev.type == "cuda" and w.m > DEVICE_FACTOR_ROWS:
        # a CPU QR of an m x r FP64 factor takes minutes at this size: the left
        # factor is drawn and orthonormalised on the device instead (FP32 QR;
        # the same distribution, other draws than the CPU path's)
        B = _orthonormal(w.n, w.r, gen).to(device=dev, dtype=work)
        gd = torch.Generator(device=dev)
        gd.manual_seed(int(w.data_seed) * 1_000_003 + 29)
        A, _ = torch.linalg.qr(torch.randn(w.m, w.r, generator=gd, dtype=torch.float32, device=dev), mode="reduced")
    else:
        A = _orthonormal(w.m, w.r, gen).to(device=dev, dtype=work)
        B = _orthonormal(w.n, w.r, gen).to(device=dev, dtype=work)
    sig = torch.as_tensor(w.sigmas(), dtype=work, device=dev)
    BS = (B * sig).T.contiguous()  # r x n
    X = out if out is not None else torch.empty(w.m, w.n, dtype=TORCH_DTYPES[w.dtype], device=dev)
    for c0 in range(0, w.m, chunk_rows):
        c1 = min(w.m, c0 + chunk_rows)
        g = torch.Generator(device=dev)
        g.manual_seed(int(w.data_seed) * 7_919 + 1 + c0 // chunk_rows)
        blk = A[c0:c1] @ BS
        if w.noise:
            blk += w.noise * torch.randn(c1 - c0, w.n, generator=g, dtype=work, device=dev)
        X[c0:c1] = blk.to(X.dtype)
    return X


def beta_rates(w: Workload) -> np.ndarray:
    """Column Bernoulli rates p_j ~ Beta(a, b), FP64, host-seeded."""
    rng = np.random.Generator(np.random.PCG64(int(w.data_seed) * 104_729 + 5))
    return rng.beta(w.extra.get("beta_a", 0.5), w.extra.get("beta_b", 9.5), size=w.n)


def binary_features(w: Workload, device="cpu", chunk_rows: int = 262144,
                    out: torch.Tensor | None = None) -> torch.Tensor:
    """X_ij = [u_ij < p_j] with p_j ~ Beta(a, b): mostly-binary sparse features
    shaped like Experiment 1's corpus.  Stored as ``TORCH_DTYPES[w.dtype]``."""
    dev = torch.device(device)
    rates = torch.as_tensor(beta_rates(w), dtype=torch.float32, device=dev)
    X = out if out is not None else torch.empty(w.m, w.n, dtype=TORCH_DTYPES[w.dtype], device=dev)
    for c0 in range(0, w.m, chunk_rows):
        c1 = min(w.m, c0 + chunk_rows)
        g = torch.Generator(device=dev)
        g.manual_seed(int(w.data_seed) * 15_485_863 + 3 + c0 // chunk_rows)
        u = torch.rand(c1 - c0, w.n, generator=g, dtype=torch.float32, device=dev)
        X[c0:c1] = (u < rates).to(torch.float32).to(X.dtype)
    return X


def generate(w: Workload, device="cpu") -> torch.Tensor:
    """The data matrix X of a workload."""
    if w.dtype == "e4m3":
        return binary_features(w, device)
    return lowrank_plus_noise(w, device)


def rank_r_exact(m: int, n: int, r: int, seed: int, dtype=torch.float64) -> tuple:
    """Noise-free X = A diag(sigma) B^T with sigma_i = 2^-i (i = 1..r).

    Returns (X, B): B spans the exact principal subspace.
    """
    gen = torch.Generator()
    gen.manual_seed(seed)
    A = _orthonormal(m, r, gen)
    B = _orthonormal(n, r, gen)
    sig = torch.tensor([2.0 ** -i for i in range(1, r + 1)], dtype=torch.float64)
    X = (A * sig) @ B.T
    return X.to(dtype), B


def serving_rows(seed: int, count: int, lo: int = 1, hi: int = 65536) -> np.ndarray:
    """Log-uniform request row counts in [lo, hi] (serving workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=count))).astype(np.int64)


SPARSE_TFIDF = {"m": 74_067, "n": 28_606, "density": 0.000513, "k": 128, "p": 169, "seed": 6, "omega_seed": 0}


def sparse_csr(m: int, n: int, density: float, seed: int) -> tuple:
    """Seeded sparse X in CSR form: (row_ptr int64 [m + 1], col int32 [nnz]
    sorted within rows, val float32 [nnz]) as CPU tensors.  Row counts are
    Poisson(density n) capped at n; the columns of a row are distinct, drawn
    with weights (j + 10)^-0.9; values 0.5 + |N(0, 1)|."""
    rng = np.random.default_rng(seed)
    counts = np.minimum(rng.poisson(density * n, m), n).astype(np.int64)
    w = (np.arange(n, dtype=np.float64) + 10.0) ** -0.9
    cdf = np.cumsum(w / w.sum())
    cols = []
    for c in counts:
        if c == 0:
            cols.append(np.zeros(0, np.int32))
            continue
        picked = np.unique(np.searchsorted(cdf, rng.random(int(c) * 2 + 4)))
        picked = picked[picked < n]
        if picked.size < c:  # top up from the uniform tail so the row has c distinct columns
            extra = rng.permutation(np.setdiff1d(np.arange(n), picked))[: int(c) - picked.size]
            picked = np.union1d(picked, extra)
        cols.append(np.sort(rng.permutation(picked)[: int(c)]).astype(np.int32))
    row_ptr = np.zeros(m + 1, np.int64)
    row_ptr[1:] = np.cumsum([c.size for c in cols])
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    val = (0.5 + np.abs(rng.standard_normal(col.size))).astype(np.float32)
    return torch.from_numpy(row_ptr), torch.from_numpy(col), torch.from_numpy(val)

"""Subspace and alignment metrics used to compare reductions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``max_sine``: largest principal-angle sine between span(A) and span(B),
  computed as the 2-norm of B - A (A^T B) (resolves angles down to ~1e-16,
  unlike sqrt(1 - cos^2)).  Prop. 2 says it is zero for V^s and V^l.
* ``chordal``: the Grassmann chordal distance ||A A^T - B B^T||_F that
  Experiment 2 uses, evaluated as sqrt(2) ||B - A (A^T B)||_F for equal
  dimensions (same value, no n x n matrices, no cancellation).
* ``procrustes_rel``: ||Y W - Y_ref||_F / ||Y_ref||_F with W the orthogonal
  k x k matrix minimising it.  Prop. 3 (equal pairwise distances) makes the
  reduced data unique only up to such a W.
* ``signaligned_rel``: the same error after only flipping column signs.
"""
from __future__ import annotations

import numpy as np


def max_sine(A: np.ndarray, B: np.ndarray) -> float:
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    R = B - A @ (A.T @ B)
    if R.size == 0:
        return 0.0
    return float(np.linalg.norm(R, 2))


def chordal(A: np.ndarray, B: np.ndarray) -> float:
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return float(np.sqrt(2.0) * np.linalg.norm(B - A @ (A.T @ B)))


def procrustes_rel(Y: np.ndarray, Yref: np.ndarray) -> float:
    Y = np.asarray(Y, np.float64)
    Yref = np.asarray(Yref, np.float64)
    u, _, vt = np.linalg.svd(Y.T @ Yref)
    W = u @ vt
    den = np.linalg.norm(Yref)
    return float(np.linalg.norm(Y @ W - Yref) / (den if den > 0 else 1.0))


def signaligned_rel(Y: np.ndarray, Yref: np.ndarray) -> float:
    Y = np.asarray(Y, np.float64)
    Yref = np.asarray(Yref, np.float64)
    s = np.sign(np.einsum("ij,ij->j", Y, Yref))
    s[s == 0] = 1.0
    den = np.linalg.norm(Yref)
    return float(np.linalg.norm(Y * s - Yref) / (den if den > 0 else 1.0))

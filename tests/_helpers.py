"""Shared test helpers: exact-QR constructions and accuracy metrics (numpy)."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U = 2.0 ** -53


def hadamard(m: int) -> np.ndarray:
    """Sylvester-Hadamard matrix H[i, j] = (-1)^popcount(i & j), m a power of 2."""
    i = np.arange(m)[:, None]
    j = np.arange(m)[None, :]
    x = i & j
    pc = np.zeros_like(x)
    while np.any(x):
        pc += x & 1
        x >>= 1
    return np.where(pc % 2 == 0, 1.0, -1.0)


def load_exact_golden(name="exact_qr_8.txt"):
    """(A, Q0, R0) of the stored exact-QR fixture."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    m, n = rows[0]
    R0 = np.array(rows[1:], dtype=np.float64)
    assert R0.shape == (n, n)
    Q0 = hadamard(m)[:, :n] / np.sqrt(m)
    A = Q0 @ R0
    return np.asfortranarray(A), Q0, R0


def exact_qr_case(m: int, n: int, seed: int, max_off: int = 3, max_log2_diag: int = 4):
    """An exact-QR input of any power-of-two m >= n: Q0 = Hadamard columns /
    sqrt(m) (a power of two when m is a power of 4), R0 integer upper
    triangular with power-of-two diagonal.  A = Q0 R0 is exact in FP64."""
    assert m & (m - 1) == 0 and n <= m
    rng = np.random.default_rng(seed)
    R0 = np.triu(rng.integers(-max_off, max_off + 1, size=(n, n))).astype(np.float64)
    np.fill_diagonal(R0, 2.0 ** rng.integers(0, max_log2_diag + 1, size=n))
    cols = np.sort(rng.choice(m, size=n, replace=False))
    Q0 = hadamard(m)[:, cols] / np.sqrt(m)
    return np.asfortranarray(Q0 @ R0), Q0, R0


def orth_err(Q) -> float:
    """||I - Q^T Q||_F (unnormalised)."""
    Q = np.asarray(Q)
    n = Q.shape[1]
    return float(np.linalg.norm(np.eye(n) - Q.T @ Q))


def resid(A, Q, R) -> float:
    """||A - Q R||_F / ||A||_F."""
    A = np.asarray(A)
    return float(np.linalg.norm(A - np.asarray(Q) @ np.asarray(R)) / np.linalg.norm(A))


def rel_diff(X, Y) -> float:
    X, Y = np.asarray(X), np.asarray(Y)
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def sign_normalised_qr(A):
    """numpy (LAPACK Householder) QR with diag(R) >= 0."""
    Q, R = np.linalg.qr(np.asarray(A))
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d, R * d[:, None]

"""Seeded synthetic test matrices (the paper's test suite, Sec. 2.2).

A = U diag(sigma) V^T with U the orthonormal Q-factor of a seeded Gaussian
m x n matrix, V a Haar-random n x n orthogonal matrix, and singular values
log-spaced from 1 down to 1/kappa:  sigma_i = kappa^(-(i-1)/(n-1)).
(Sec. 2.2 describes the diagonal as (1, s^(1/(n-1)), ..., s) with the
condition number controlled by s; the reading used here is s = 1/kappa, so
that cond(A) = kappa exactly.)

This module holds no CholeskyQR arithmetic.  It is shared by the CPU oracle
tests and the GPU tests and benchmarks, which is the only thing the two
sides share.  Small matrices are generated on the CPU with numpy (PCG64),
so both sides see identical bits; large ones are generated on the GPU with
torch's generator and library QR/GEMM.
"""
from __future__ import annotations

import numpy as np

# Seeds of the five workload configurations (seed = 1000 + index) and of the
# batched configuration's per-matrix draws.
SEED_BASE = 1000
SEED_BATCH = 4000


def sigma(n: int, kappa: float) -> np.ndarray:
    """Log-spaced singular values 1 = s_1 >= ... >= s_n = 1/kappa."""
    if n == 1:
        return np.ones(1)
    return np.power(float(kappa), -np.arange(n, dtype=np.float64) / (n - 1))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix: Q of a Gaussian matrix with
    the signs fixed by diag(R) (Mezzadri, Notices AMS 54 (2007))."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def orthonormal_columns(m: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """Q-factor (m x n) of a Gaussian m x n matrix."""
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    return Q


def make_test_matrix(m: int, n: int, kappa: float, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T (column-major FP64 numpy array), CPU, seeded."""
    rng = np.random.default_rng(seed)
    U = orthonormal_columns(m, n, rng)
    V = haar_orthogonal(n, rng)
    A = (U * sigma(n, kappa)) @ V.T
    return np.asfortranarray(A)


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((m, n)))


def make_test_matrix_cuda(m: int, n: int, kappa: float, seed: int, device="cuda", chunk_rows: int = 1 << 20):
    """A = U diag(sigma) V^T generated on the GPU (for sizes the CPU cannot
    hold or generate quickly).  Returns a column-major torch FP64 tensor.

    U is the Q-factor (torch.linalg.qr, Householder) of a Gaussian drawn from
    a torch CUDA generator seeded with `seed`; V is Haar (n x n, CPU numpy,
    same seed).  The product is formed in row chunks to bound the extra
    memory to one chunk.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    G = torch.randn((n, m), generator=g, dtype=torch.float64, device=device).t()  # column-major m x n
    U = torch.linalg.qr(G, mode="reduced").Q
    del G
    if U.stride(0) != 1:
        U = U.t().contiguous().t()
    rng = np.random.default_rng(seed)
    V = torch.from_numpy(haar_orthogonal(n, rng)).to(device)
    s = torch.from_numpy(sigma(n, kappa)).to(device)
    SVt = (s[:, None] * V.t()).contiguous()  # diag(sigma) V^T, so A = U @ SVt
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        U[r0:r1] = U[r0:r1] @ SVt
    return U


def batch_specs(count: int = 512, seed: int = SEED_BATCH, m_range=(2000, 200000), n_choices=(16, 32, 64, 128),
                log10_kappa=(2.0, 15.0)):
    """Per-matrix (m, n, kappa, seed) of the batched workload: m uniform in
    m_range, n uniform over n_choices, kappa log-uniform; matrix i is seeded
    with seed + 1 + i."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ns = rng.choice(np.asarray(n_choices), size=count)
    ks = np.power(10.0, rng.uniform(log10_kappa[0], log10_kappa[1], size=count))
    return [(int(ms[i]), int(ns[i]), float(ks[i]), seed + 1 + i) for i in range(count)]

"""The seeded input recipe (Sec. 2.2 construction), checked on the CPU:
A = U diag(sigma) V^T with orthonormal U, orthogonal V and log-spaced
singular values, so that cond(A) = kappa; the large-matrix generator (torch,
run here on the CPU device) gives the same spectrum; the batched workload's
draws stay in their ranges and are reproducible."""
import numpy as np
import pytest

from testmatrices import batch_specs, haar_orthogonal, make_test_matrix, orthonormal_columns, sigma

torch = pytest.importorskip("torch")


def test_haar_and_orthonormal_factors():
    rng = np.random.default_rng(3)
    V = haar_orthogonal(40, rng)
    assert np.linalg.norm(V.T @ V - np.eye(40)) < 1e-13
    U = orthonormal_columns(500, 40, rng)
    assert np.linalg.norm(U.T @ U - np.eye(40)) < 1e-13


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e15])
def test_singular_values_follow_the_recipe(kappa):
    A = make_test_matrix(400, 12, kappa, seed=4)
    sv = np.linalg.svd(A, compute_uv=False)
    # relative accuracy of the smallest singular values is limited by u / sigma_min
    assert np.allclose(sv[:4], sigma(12, kappa)[:4], rtol=1e-12, atol=0)
    assert abs(sv[0] - 1.0) < 1e-13 and sv[-1] > 0
    if kappa <= 1e8:
        assert abs(sv[0] / sv[-1] / kappa - 1) < 1e-6


def test_seeded_and_reproducible():
    assert np.array_equal(make_test_matrix(100, 6, 1e5, seed=9), make_test_matrix(100, 6, 1e5, seed=9))
    assert not np.array_equal(make_test_matrix(100, 6, 1e5, seed=9), make_test_matrix(100, 6, 1e5, seed=10))
    assert np.isfortran(make_test_matrix(100, 6, 1e5, seed=9))


def test_large_matrix_generator_spectrum():
    from testmatrices import make_test_matrix_cuda

    A = make_test_matrix_cuda(3000, 16, 1e6, seed=5, device="cpu", chunk_rows=1000)
    assert A.stride(0) == 1 and A.stride(1) == 3000  # column-major
    sv = torch.linalg.svdvals(A).numpy()
    assert np.allclose(sv, sigma(16, 1e6), rtol=1e-9, atol=0)


def test_batch_specs_ranges_and_reproducibility():
    specs = batch_specs(512)
    assert specs == batch_specs(512)
    ms = np.array([s[0] for s in specs])
    ns = np.array([s[1] for s in specs])
    ks = np.array([s[2] for s in specs])
    seeds = [s[3] for s in specs]
    assert ms.min() >= 2000 and ms.max() <= 200000
    assert set(ns.tolist()) <= {16, 32, 64, 128} and len(set(ns.tolist())) == 4
    assert ks.min() >= 1e2 * (1 - 1e-12) and ks.max() <= 1e15 * (1 + 1e-12)
    assert seeds == list(range(4001, 4001 + 512))

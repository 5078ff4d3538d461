"""The 2^23 x 1024 mCQR2GS factorisation (kappa = 1e15, b = 128, the
benchmark's matrix) compared with the CPU oracle on the same input.

Not a pytest test (the oracle needs about 12 minutes on 16 host cores and
69 GB of host memory): run as

    python tests/headline_oracle_comparison.py [--out FILE]

It prints one JSON object:
  * the GPU's ||I - Q^T Q||_F and ||A - Q R||_F / ||A||_F (torch FP64 GEMMs
    over row chunks) and the same two norms of the oracle's factors;
  * ||R_gpu - R_oracle||_F / ||R_oracle||_F over all of R;
  * max |Q_gpu - Q_oracle| over 65,536 seeded sampled rows (and that
    maximum relative to max |Q| on those rows).
At kappa = 1e15 the element-wise differences are reported, not asserted:
R's forward error grows like kappa u, so only the norms have a bound.
The test matrix is regenerated on the GPU for the oracle's norms, and a
checksum of sampled rows confirms it is the same matrix.
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_2405_04237_gb300 as P  # noqa: E402
from testmatrices import make_test_matrix_cuda  # noqa: E402

M, N, KAPPA, SEED, B = 1 << 23, 1024, 1e15, 1002, 128
SAMPLE_ROWS, SAMPLE_SEED = 65536, 11


def norms(A, Q, R, chunk=1 << 20):
    """||I - Q^T Q||_F and ||A - Q R||_F / ||A||_F (Q may be a host array)."""
    n = R.shape[0]
    G = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    r2 = torch.zeros((), dtype=torch.float64, device="cuda")
    a2 = torch.zeros((), dtype=torch.float64, device="cuda")
    for r0 in range(0, A.shape[0], chunk):
        r1 = min(A.shape[0], r0 + chunk)
        Qc = Q[r0:r1] if torch.is_tensor(Q) else torch.from_numpy(np.ascontiguousarray(Q[r0:r1])).cuda()
        G += Qc.t() @ Qc
        D = A[r0:r1] - Qc @ R
        r2 += (D * D).sum()
        a2 += (A[r0:r1] ** 2).sum()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - G).item()
    return orth, (r2.sqrt() / a2.sqrt()).item()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    rows = np.sort(np.random.default_rng(SAMPLE_SEED).choice(M, SAMPLE_ROWS, replace=False))
    idx = torch.from_numpy(rows).cuda()
    out = {"m": M, "n": N, "kappa": KAPPA, "panel_b": B, "seed": SEED, "sample_rows": SAMPLE_ROWS,
           "oracle_threads": oracle.num_threads()}

    A = make_test_matrix_cuda(M, N, KAPPA, SEED)
    check_rows = A.index_select(0, idx[:64]).cpu().numpy()
    Q = P.empty_colmajor(M, N, "cuda")
    R = P.empty_colmajor(N, N, "cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.factor(A, B, "mcqr2gs", out=(Q, R))
    torch.cuda.synchronize()
    out["gpu_seconds"] = time.perf_counter() - t0
    out["gpu_orth_fro"], out["gpu_resid_rel"] = norms(A, Q, R)
    Qs = Q.index_select(0, idx).cpu().numpy()
    Rg = R.cpu().numpy()
    del Q, R
    A_host = np.asfortranarray(A.cpu().numpy())  # the column-major device matrix, as a Fortran-ordered array
    del A
    torch.cuda.empty_cache()

    t0 = time.perf_counter()
    Qo, Ro = oracle.mcqr2gs(A_host, B, inplace=True)  # Qo is A_host, overwritten
    out["oracle_seconds"] = time.perf_counter() - t0
    out["R_rel_diff_fro"] = float(np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro))
    dq = np.abs(Qs - Qo[rows])
    out["Q_sampled_max_abs_diff"] = float(dq.max())
    out["Q_sampled_max_abs_diff_rel_to_max_Q"] = float(dq.max() / np.abs(Qs).max())

    A = make_test_matrix_cuda(M, N, KAPPA, SEED)  # regenerated for the oracle's norms
    out["regenerated_matrix_identical"] = bool(np.array_equal(A.index_select(0, idx[:64]).cpu().numpy(),
                                                              check_rows))
    out["oracle_orth_fro"], out["oracle_resid_rel"] = norms(A, Qo, torch.from_numpy(Ro).cuda(), chunk=1 << 18)
    text = json.dumps(out, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()

"""Writes fullsize_oracle_error.txt: the final relative error of the FP64
oracle's TTNN on the bench workload (64^5 tensor 1/sum(x) on [1,2]^5 in
binary64, balanced binary tree, r = 20, p = 10, DRM seed 2024), measured on
20000 seeded sample entries against the exact values.  Calls only oracle/ and
the seeded generators; needs ~40 GB of host memory and a few minutes.

    python tests/golden/make_fullsize_oracle_error.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import workloads as W  # noqa: E402
from oracle import ttnn as O  # noqa: E402
from oracle.tree import Tree  # noqa: E402

D, N, RANK, OVER, SEED = 5, 64, 20, 10, 2024
SAMPLES, SAMPLE_SEED = 20000, 77


def sample_indices():
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.stack([rng.integers(0, N, size=SAMPLES) for _ in range(D)], axis=1)


def exact_values(idx):
    return 1.0 / (1.0 + idx / (N - 1)).sum(axis=1)


def main():
    tr = W.balanced_binary(D)
    n = len(tr[0])
    t = Tree(tr[0], tr[1], [N] * D, [RANK] * n, [OVER] * n, tr[2])
    T = W.inv_sum(D, N)
    cores, _ = O.ttnn(T, t, SEED, "f64")
    R = O.reconstruct(t, cores)
    idx = sample_indices()
    approx = R[tuple(idx.T)]
    ex = exact_values(idx)
    err = float(np.linalg.norm(approx - ex) / np.linalg.norm(ex))
    full = float(np.linalg.norm(R - T) / np.linalg.norm(T))
    with open(os.path.join(HERE, "fullsize_oracle_error.txt"), "w") as f:
        f.write("# FP64 oracle TTNN, 64^5 inv-sum, r=20 p=10 seed 2024 (make_fullsize_oracle_error.py)\n")
        f.write(f"sampled_rel_error: {err:.6e}\n")
        f.write(f"full_rel_error: {full:.6e}\n")
    print(err, full)


if __name__ == "__main__":
    main()

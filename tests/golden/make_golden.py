"""Writes tests/golden/lattice_ties.json from the CPU oracle only.

The case is a small integer lattice (spacing 0.5, exactly representable)
with queries on lattice points, cell centres and edge midpoints, so almost
every neighbour distance is an exact tie: it fixes the (d2, index) order,
the pinned binary32 d2 values and the binary64 covariances (raw and
plane-regularised) of Sec. III-C1's per-point Gaussians for a reader to
check by hand.  The paper prints no worked example, so these values come
from the oracle, which tests/test_oracle_pins.py pins independently.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def lattice_case():
    g = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(3), indexing="ij"), -1)
    p = (g.reshape(-1, 3) * 0.5).astype(np.float32)
    p = p[np.random.default_rng(2024).permutation(len(p))]
    q = np.array([[1.0, 1.0, 0.5], [1.25, 1.25, 0.25], [0.25, 0.0, 0.0], [2.5, 2.0, 1.0],
                  [-0.5, -0.5, -0.5], [1.25, 1.0, 0.5]], np.float32)
    return p, q


def main():
    p, q = lattice_case()
    k = 10
    idx, d2 = oracle.knn_brute(q, p, k)
    out = {
        "about": "6x5x3 lattice, spacing 0.5, shuffled with PCG64 seed 2024; k=10; written by make_golden.py from the CPU oracle",
        "points": p.tolist(),
        "queries": q.tolist(),
        "k": k,
        "idx": idx.tolist(),
        "d2": d2.tolist(),
        "cov_raw": oracle.cov(p, idx, -1.0).tolist(),
        "cov_reg_eps_0.01": oracle.cov(p, idx, 0.01).tolist(),
    }
    with open(os.path.join(HERE, "lattice_ties.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()

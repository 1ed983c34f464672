"""The committed lattice fixture (tests/golden/lattice_ties.json, written
by tests/golden/make_golden.py from the oracle alone): the oracle must keep
reproducing it, its first row must match the lattice's closed form, and
the CUDA path must reproduce it bit for bit (idx, d2) and within the
covariance bar."""
import json
import os

import numpy as np
import pytest

import oracle
from tests import helpers as H

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "lattice_ties.json")))
P = np.array(G["points"], np.float32)
Q = np.array(G["queries"], np.float32)
K = G["k"]


def test_oracle_reproduces_golden():
    idx, d2 = oracle.knn_brute(Q, P, K)
    np.testing.assert_array_equal(idx, np.array(G["idx"], np.int32))
    np.testing.assert_array_equal(d2, np.array(G["d2"], np.float32))
    np.testing.assert_allclose(oracle.cov(P, idx, -1.0), np.array(G["cov_raw"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.cov(P, idx, 0.01), np.array(G["cov_reg_eps_0.01"]), rtol=0, atol=1e-13)


def test_golden_first_row_closed_form():
    # query 0 sits on a lattice point away from the border: itself, its six
    # face neighbours (d2 = 0.25) and then edge neighbours (d2 = 0.5), with
    # ties in ascending index
    d2 = np.array(G["d2"][0])
    np.testing.assert_array_equal(d2, [0.0] + [0.25] * 6 + [0.5] * 3)
    idx = np.array(G["idx"][0])
    assert (np.diff(idx[1:7]) > 0).all() and (np.diff(idx[7:]) > 0).all()
    assert np.allclose(P[idx[0]], Q[0])


@pytest.mark.gpu
def test_gpu_reproduces_golden(gpu_lib):
    torch = pytest.importorskip("torch")
    t = gpu_lib.Target(torch.from_numpy(P).cuda(), cell_size=0.5)
    i, d, c = t.knn_cov(torch.from_numpy(Q).cuda(), K, -1.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(i.cpu().numpy(), np.array(G["idx"], np.int32))
    np.testing.assert_array_equal(d.cpu().numpy(), np.array(G["d2"], np.float32))
    H.check_raw_cov(c.cpu().numpy(), np.array(G["cov_raw"]))
    t.close()

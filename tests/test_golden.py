"""Stored expected values (tests/golden/small_k.json, written by tests/golden/make_golden.py from
the oracle alone) pinned against an independent route, LAPACK's generalized symmetric eigensolver
(scipy.linalg.eigh(A, B)), and re-derived by the oracle (a change in the oracle's arithmetic shows
here).  The GPU path is checked against the same stored values."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from gen import workload
from oracle import core

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "small_k.json")) as f:
        g = json.load(f)
    p = workload("small", seed=0)
    return g, p, p.A().toarray(), p.B().toarray()


def test_stored_values_against_lapack(golden):
    g, p, A, B = golden
    assert (g["n"], g["k"]) == (p.n, p.k)
    w = sla.eigh(A, B, eigvals_only=True)
    nrm = g["norm_a_inf"]
    for i, v in g["lambda"].items():
        assert abs(w[int(i) - 1] - v) <= 1e-12 * nrm, i
    for s, nu in zip(g["shifts"], g["nu"]):
        assert int(np.count_nonzero(w < s)) == nu
        d = np.abs(w - s).min()
        assert d > 1e-8 * nrm                     # certified: no eigenvalue near the shift


def test_oracle_reproduces_stored_values(golden):
    g, p, A, B = golden
    lam, _ = core.gen_eig(A, B)
    for i, v in g["lambda"].items():
        assert abs(lam[int(i) - 1] - v) <= 1e-13 * g["norm_a_inf"], i
    assert [core.dense_nu(A, B, s) for s in g["shifts"]] == g["nu"]


@pytest.mark.gpu
def test_gpu_path_against_stored_values(golden):
    from tests.gpu_util import require_gpu
    kep = require_gpu()
    g, p, A, B = golden
    with kep.Problem.from_pencil(p) as P:
        for s, nu in zip(g["shifts"], g["nu"]):
            assert P.factor(s).neg == nu
        lam, x, rep = P.kth_eigenpair(g["k"])
    assert abs(lam - g["lambda"][str(g["k"])]) <= 1e-10 * g["norm_a_inf"]
    assert rep["rel_res"] < 1e-10

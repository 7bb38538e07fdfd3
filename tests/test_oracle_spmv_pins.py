"""Pins of the SpMV oracle (y = A x, CSR with values) against facts outside its own loop: a dense
matrix product, identity and permutation matrices, row sums, and linearity."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle


def _dense(n, rp, ci, vals):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, ci[k]] += vals[k]
    return A


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_dense_product(seed):
    g = gg.random_small(150, 1200, seed)
    rp, ci = g.numpy()
    vals = gg.edge_values(g, seed=seed).numpy().astype(np.float64)
    x = np.random.default_rng(seed).standard_normal(g.V)
    want = _dense(g.V, rp, ci, vals) @ x
    np.testing.assert_allclose(oracle.spmv(g.V, rp, ci, vals, x), want, rtol=1e-12, atol=1e-12)


def test_identity_and_permutation():
    n = 64
    x = np.random.default_rng(0).standard_normal(n)
    rp = np.arange(n + 1, dtype=np.int32)
    eye = np.arange(n, dtype=np.int32)
    np.testing.assert_array_equal(oracle.spmv(n, rp, eye, np.ones(n), x), x)
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    np.testing.assert_array_equal(oracle.spmv(n, rp, perm, np.ones(n), x), x[perm])


def test_row_counts_and_empty_rows():
    g = gg.powerlaw_config(500, 6, 2.2, seed=3)
    rp, ci = g.numpy()
    y = oracle.spmv(g.V, rp, ci, np.ones(g.E), np.ones(g.V))
    np.testing.assert_array_equal(y, np.diff(rp).astype(np.float64))
    e = gg.empty_graph(7)
    rp, ci = e.numpy()
    assert np.all(oracle.spmv(7, rp, ci, np.zeros(0), np.ones(7)) == 0.0)


def test_linearity_and_unweighted_gather():
    """A(a x + b z) = a Ax + b Az; with unit values on G^T it is the in-edge sum of Alg. 1."""
    g = gg.rmat(10)
    rp, ci = g.numpy()
    vals = gg.edge_values(g).numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    x, z = rng.standard_normal(g.V), rng.standard_normal(g.V)
    lhs = oracle.spmv(g.V, rp, ci, vals, 2.0 * x - 3.0 * z)
    rhs = 2.0 * oracle.spmv(g.V, rp, ci, vals, x) - 3.0 * oracle.spmv(g.V, rp, ci, vals, z)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-10)
    trp, tci = oracle.transpose(g.V, rp, ci)
    y = oracle.spmv(g.V, trp, tci, np.ones(g.E), x)
    want = np.zeros(g.V)
    np.add.at(want, ci, x[np.repeat(np.arange(g.V), np.diff(rp))])
    np.testing.assert_allclose(y, want, rtol=1e-12, atol=1e-12)


def test_edge_values_are_seeded_and_in_range():
    g = gg.rmat(9)
    a, b = gg.edge_values(g, seed=4), gg.edge_values(g, seed=4)
    assert torch.equal(a, b) and a.dtype == torch.float32 and a.numel() == g.E
    assert float(a.min()) >= -1.0 and float(a.max()) < 1.0
    assert not torch.equal(a, gg.edge_values(g, seed=5))

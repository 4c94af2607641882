"""The seeded generators: shapes, row sums, distinct sorted successors, determinism."""
import numpy as np

import mdpgen


def test_csr_rows_are_distributions_with_distinct_sorted_successors():
    m = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.9, seed=3)
    assert m.uniform_k() == 16 and m.nnz == 3000 * 4 * 16
    rs = np.add.reduceat(m.prob.astype(np.float64), m.row_ptr[:-1])
    assert np.max(np.abs(rs - 1)) < 1e-6
    c = m.col.reshape(-1, 16)
    assert np.all(np.diff(c, axis=1) > 0) and c.min() >= 0 and c.max() < 3000
    m2 = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.9, seed=3)
    assert np.array_equal(m.col, m2.col) and np.array_equal(m.prob, m2.prob)


def test_softmax_rows_and_logits():
    m = mdpgen.csr_uniform_k(500, 3, 8, gamma=0.9, seed=1, prob_kind="softmax")
    z = m.logits.astype(np.float64).reshape(-1, 8)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    assert np.max(np.abs(m.prob.reshape(-1, 8) - e / e.sum(axis=1, keepdims=True))) < 1e-7


def test_dense_and_batched():
    d = mdpgen.dense_dirichlet(64, 3, alpha=0.1, gamma=0.99, seed=2, cost_dist="normal")
    assert d.P.shape == (64, 3, 64)
    assert np.max(np.abs(d.P.astype(np.float64).sum(axis=2) - 1)) < 1e-6
    b = mdpgen.batched_uneven(10, 256, 4096, 16, seed=5)
    assert len(b) == 10 and all(256 <= x.n <= 4096 and 2 <= x.m <= 16 and 0.9 <= x.gamma <= 0.99 for x in b)
    assert len({x.n for x in b}) > 1

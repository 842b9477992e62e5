"""Pins of the oracle's particle -> field transfers of Sec. 2.7 (iv) and (v).

(iv) shape-function-weighted vertex averages (reading R17):
  - particles sitting exactly on the vertices return the vertex values
    exactly (one weight 1, the others 0): pins the vertex numbering;
  - constant properties are reproduced; the weights are a partition of
    unity, so the weight sums add up to N and sum_v avg_v w_v = sum_i p_i;
  - a hand-computed one-cell case.
(v) per-cell linear least squares in reference coordinates (reading R18):
  - data linear in x-hat is reproduced exactly;
  - the residual is orthogonal to the design matrix's columns;
  - the coefficients agree with an SVD least-squares solver (numpy.lstsq)
    within the conditioning of the cell's normal matrix;
  - cells with at most dim particles, or degenerate ones, fall back to the
    mean; empty cells get the fill value.
"""
import itertools

import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W


def _store(O, n, ppc, seed):
    X = W.jittered_vertices(n, seed)
    m = O.Mesh(n, X)
    p = O.seed_particles(m, uniform_count=ppc, seed=seed)
    return m, p


@pytest.mark.parametrize("n", [(3, 2), (2, 3, 2)])
def test_vertex_average_particles_on_vertices(oracle_mod, n):
    O = oracle_mod
    dim = len(n)
    X = W.jittered_vertices(n, 4)
    m = O.Mesh(n, X)
    nv = [v + 1 for v in n]
    f = lambda v: 3.0 * v[0] - 2.0 * v[1] + (0.5 * v[2] if dim == 3 else 0.0) + 0.25
    cells, xh, vals = [], [], []
    for v in itertools.product(*[range(k) for k in nv]):
        # the lowest-index cell holding vertex v, and v's local corner there
        c = [min(v[a], n[a] - 1) for a in range(dim)]
        K = c[0] + n[0] * (c[1] + (n[1] * c[2] if dim == 3 else 0))
        cells.append(K)
        xh.append([float(v[a] - c[a]) for a in range(dim)])
        vals.append(f(v))
    order = np.argsort(cells, kind="stable")
    cells = np.array(cells)[order]
    xh = np.array(xh)[order]
    vals = np.array(vals)[order]
    avg, w = O.vertex_average(m, cells, xh, vals, empty_fill=-7.0)
    want = np.array([f(v) for v in itertools.product(*[range(k) for k in nv])])
    # vertex index i + nv0 (j + nv1 k) enumerates with the first axis fastest
    want = want.reshape([k for k in nv]).transpose(list(range(dim))[::-1]).reshape(-1)
    np.testing.assert_array_equal(w, np.ones_like(w))
    np.testing.assert_array_equal(avg, want)


def test_vertex_average_one_cell_by_hand(oracle_mod):
    O = oracle_mod
    X = np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0]])
    m = O.Mesh((1, 1), X)
    xh = np.array([[0.25, 0.5], [0.75, 0.0]])
    v = np.array([2.0, 6.0])
    avg, w = O.vertex_average(m, np.zeros(2, np.int64), xh, v)
    # corner weights: (1-s)(1-t), s(1-t), (1-s)t, st
    w1 = np.array([0.375, 0.125, 0.375, 0.125])
    w2 = np.array([0.25, 0.75, 0.0, 0.0])
    np.testing.assert_allclose(w, w1 + w2, rtol=0, atol=1e-16)
    np.testing.assert_allclose(avg, (2.0 * w1 + 6.0 * w2) / (w1 + w2), rtol=1e-15)


@pytest.mark.parametrize("n", [(6, 5), (4, 3, 3)])
def test_vertex_average_constant_and_conservation(oracle_mod, n):
    O = oracle_mod
    m, p = _store(O, n, 5, 9)
    c = 1.7
    avg, w = O.vertex_average(m, p.cell, p.xhat, np.full(p.n, c), empty_fill=0.0)
    assert (w > 0).all()
    np.testing.assert_allclose(avg, c, rtol=4e-16 * 8)
    assert abs(w.sum() - p.n) < 1e-11 * p.n
    vals = np.random.default_rng(2).uniform(-1, 1, p.n)
    avg, w = O.vertex_average(m, p.cell, p.xhat, vals)
    assert abs((avg * w).sum() - vals.sum()) < 1e-12 * np.abs(vals).sum()
    lo, hi = vals.min(), vals.max()
    assert (avg >= lo - 1e-15).all() and (avg <= hi + 1e-15).all()  # a convex combination


def test_vertex_average_empty_support(oracle_mod):
    O = oracle_mod
    m = O.Mesh((3, 1), W.uniform_vertices((3, 1)))
    avg, w = O.vertex_average(m, np.array([0]), np.array([[0.5, 0.5]]), np.array([4.0]), empty_fill=-1.0)
    np.testing.assert_array_equal(w, [0.25, 0.25, 0, 0, 0.25, 0.25, 0, 0])
    np.testing.assert_array_equal(avg, [4.0, 4.0, -1, -1, 4.0, 4.0, -1, -1])


@pytest.mark.parametrize("n", [(5, 4), (3, 3, 3)])
def test_lsq_reproduces_linear_data(oracle_mod, n):
    O = oracle_mod
    dim = len(n)
    m, p = _store(O, n, 7, 3)
    g = np.random.default_rng(5)
    C = m.ncells
    a = g.uniform(-2, 2, (C, dim + 1))
    vals = a[p.cell, 0] + ((p.xhat - 0.5) * a[p.cell, 1:]).sum(axis=1)
    coef, cnt = O.cell_lsq_linear(m, p.cell, p.xhat, vals)
    np.testing.assert_array_equal(cnt, np.full(C, 7))
    np.testing.assert_allclose(coef, a, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [(5, 4), (3, 3, 3)])
def test_lsq_normal_equations_and_svd(oracle_mod, n):
    O = oracle_mod
    dim = len(n)
    g = np.random.default_rng(8)
    X = W.jittered_vertices(n, 6)
    m = O.Mesh(n, X)
    per = g.integers(dim + 1, 12, size=m.ncells).astype(np.uint32)
    p = O.seed_particles(m, per_cell=per, seed=6)
    vals = np.sin(7 * p.x[:, 0]) + p.x[:, 1] ** 2
    coef, cnt = O.cell_lsq_linear(m, p.cell, p.xhat, vals)
    for K in range(m.ncells):
        sel = p.cell == K
        A = np.hstack([np.ones((sel.sum(), 1)), p.xhat[sel] - 0.5])
        r = A @ coef[K] - vals[sel]
        # first-order optimality: the residual is orthogonal to every column
        assert np.abs(A.T @ r).max() <= 1e-13 * np.abs(A).sum(axis=0).max() * max(1.0, np.abs(vals[sel]).max())
        ref = np.linalg.lstsq(A, vals[sel], rcond=None)[0]
        kappa = np.linalg.cond(A.T @ A)
        assert np.abs(coef[K] - ref).max() <= 64 * 2.2e-16 * kappa * max(1.0, np.abs(ref).max())


def test_lsq_fallbacks(oracle_mod):
    O = oracle_mod
    m = O.Mesh((4, 1), W.uniform_vertices((4, 1)))
    # cell 0: 2 particles (<= dim): mean; cell 1: empty; cell 2: 5 particles at
    # the same point (degenerate): mean; cell 3: 3 generic particles: exact fit
    cell = np.array([0, 0, 2, 2, 2, 2, 2, 3, 3, 3])
    xh = np.array([[0.1, 0.2], [0.7, 0.9]] + [[0.3, 0.6]] * 5 + [[0.1, 0.1], [0.9, 0.2], [0.4, 0.8]])
    v = np.array([1.0, 3.0, 2.0, 4.0, 6.0, 8.0, 10.0, 0.0, 0.0, 0.0])
    v[7:] = 0.5 + 2.0 * (xh[7:, 0] - 0.5) - 1.0 * (xh[7:, 1] - 0.5)
    coef, cnt = O.cell_lsq_linear(m, cell, xh, v, empty_fill=-9.0)
    np.testing.assert_array_equal(cnt, [2, 0, 5, 3])
    np.testing.assert_array_equal(coef[0], [2.0, 0.0, 0.0])
    np.testing.assert_array_equal(coef[1], [-9.0, 0.0, 0.0])
    np.testing.assert_array_equal(coef[2], [6.0, 0.0, 0.0])
    np.testing.assert_allclose(coef[3], [0.5, 2.0, -1.0], rtol=0, atol=1e-14)

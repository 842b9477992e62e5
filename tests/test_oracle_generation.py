"""Pins of the oracle's generation with a density (Sec. 2.2): cell weights,
per-cell counts, in-cell Metropolis-Hastings sampling, and prescribed
locations.

- Cell weights: with rho = 1 the weights are the cell volumes and add up to
  the unit domain's volume; with rho = the vertices' x coordinate (which the
  (bi/tri)linear interpolant reproduces exactly) they add up to
  int_[0,1]^d x = 1/2.  Both fail for a missing |det J| or a rule that is
  not exact for degree 3.
- Counts: the draws follow the published SplitMix64 outputs (pinned by the
  golden vector) and the "first accumulated weight above r" rule, checked on
  a hand case; zero-weight cells get nothing; the counts add up to N and fit
  N w_K / W (chi-square, fixed seed).
- MH: with a constant pulled-back density every proposal is accepted, so the
  particles are exactly the proposals of steps J, 2J, ...; with a density
  linear in x-hat_0 the samples' mean matches the closed form.
- Import: cell-centre points land in their cell with x-hat = 1/2; points
  outside are skipped; ids follow the input order of the points found.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W


def _u(O, seed, i):
    return (O.splitmix64(seed, i) >> 11) * 2.0**-53


@pytest.mark.parametrize("n", [(7, 5), (4, 3, 5)])
def test_cell_weights_volume_and_first_moment(oracle_mod, n):
    O = oracle_mod
    X = W.jittered_vertices(n, 13)
    m = O.Mesh(n, X)
    w = O.cell_weights(m, np.ones(X.shape[1]))
    assert (w > 0).all()
    assert abs(w.sum() - 1.0) < 1e-14
    w1 = O.cell_weights(m, X[0].copy())
    assert abs(w1.sum() - 0.5) < 1e-14
    # a midpoint rule would miss both on jittered cells: make sure they are curved
    one = O.cell_weights(m, np.ones(X.shape[1]))
    assert np.abs(one - 1.0 / m.ncells).max() > 1e-4


def test_cell_weights_affine_by_hand(oracle_mod):
    O = oracle_mod
    # one parallelogram cell: (0,0), (2,0), (0.5,1), (2.5,1): area 2
    X = np.array([[0.0, 2.0, 0.5, 2.5], [0.0, 0.0, 1.0, 1.0]])
    m = O.Mesh((1, 1), X)
    # rho = 1 + y at the vertices -> int (1 + y) over the parallelogram = 2 * (1 + 1/2)
    w = O.cell_weights(m, 1.0 + X[1])
    assert abs(w[0] - 3.0) < 1e-15


def test_draw_counts_hand_case(oracle_mod):
    O = oracle_mod
    w = np.array([1.0, 0.0, 3.0, 0.0])
    seed, N = 77, 400
    counts = O.draw_cell_counts(w, N, seed)
    r = np.array([4.0 * _u(O, seed, i) for i in range(N)])
    np.testing.assert_array_equal(counts, [int((r < 1.0).sum()), 0, int((r >= 1.0).sum()), 0])


def test_draw_counts_statistics(oracle_mod):
    O = oracle_mod
    g = np.random.default_rng(4)
    C = 200
    w = g.uniform(0.0, 1.0, C) ** 3
    w[::9] = 0.0
    N = 100000
    counts = O.draw_cell_counts(w, N, 12345)
    assert counts.sum() == N
    assert (counts[w == 0] == 0).all()
    e = N * w / w.sum()
    pos = e > 0
    chi2 = (((counts[pos] - e[pos]) ** 2) / e[pos]).sum()
    dof = pos.sum() - 1
    # chi-square with ~180 degrees of freedom: mean dof, sd sqrt(2 dof)
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)


def test_mh_constant_density_takes_every_proposal(oracle_mod):
    O = oracle_mod
    n = (3, 2, 2)
    X = W.uniform_vertices(n)
    X[0] = X[0] * 1.5 + 0.3 * X[1]  # affine: det J constant
    m = O.Mesh(n, X)
    per = np.array([2, 0, 3, 1, 0, 4, 2, 2, 1, 0, 3, 1], dtype=np.uint32)
    J, seed = 5, 99
    p = O.seed_particles_mh(m, per, np.full(X.shape[1], 2.5), J, seed, first_id=10)
    assert p.n == per.sum()
    np.testing.assert_array_equal(p.cell, np.repeat(np.arange(12), per))
    np.testing.assert_array_equal(p.id, 10 + np.arange(p.n, dtype=np.uint64))
    for g in range(p.n):
        step = J * g + (J - 1)  # the chain's global step that produced particle g
        want = [_u(O, seed, step * 4 + j) for j in range(3)]
        np.testing.assert_array_equal(p.xhat[g], want)
        np.testing.assert_allclose(p.x[g], m.phi(int(p.cell[g]), p.xhat[g]), rtol=0, atol=0)


def test_mh_linear_density_moments(oracle_mod):
    O = oracle_mod
    n = (8, 8, 8)
    X = W.uniform_vertices(n)
    m = O.Mesh(n, X)
    # rho = 1 + 3 t_0 inside every cell (t_0 the cell-local x-hat_0)
    nv = [k + 1 for k in n]
    i0 = np.arange(X.shape[1]) % nv[0]
    rho = np.where(i0 % 2 == 0, 1.0, 4.0)  # cells alternate orientation along x
    per = np.full(m.ncells, 20, dtype=np.uint32)
    p = O.seed_particles_mh(m, per, rho, 8, 2024)
    ci = p.cell % n[0]
    t0 = np.where(ci % 2 == 0, p.xhat[:, 0], 1.0 - p.xhat[:, 0])  # the coordinate along increasing rho
    # density (1 + 3t) / 2.5 on [0,1]: mean 0.6, second moment 0.43
    assert abs(t0.mean() - 0.6) < 0.01
    assert abs((t0 ** 2).mean() - (1 / 3 + 3 / 4) / 2.5) < 0.01
    assert abs(p.xhat[:, 1].mean() - 0.5) < 0.01 and abs(p.xhat[:, 2].mean() - 0.5) < 0.01
    for K in (0, 100, 511):  # each particle lies in its cell
        for g in np.flatnonzero(p.cell == K)[:3]:
            ok, t = m.inside(K, p.x[g])
            assert ok


@pytest.mark.parametrize("n", [(5, 4), (3, 4, 2)])
def test_import_points(oracle_mod, n):
    O = oracle_mod
    dim = len(n)
    X = W.jittered_vertices(n, 21)
    m = O.Mesh(n, X)
    C = m.ncells
    centres = np.array([m.phi(K, np.full(dim, 0.5)) for K in range(C)])
    outside = np.full((4, dim), 0.5)
    outside[:, 0] = [-0.2, 1.3, -1e-3, 1.0 + 1e-3]
    g = np.random.default_rng(1)
    order = g.permutation(C + 4)
    pts = np.concatenate([centres, outside])[order]
    p = O.import_points(m, pts, first_id=100)
    assert p.n == C
    # ids follow the input order of the points that were found
    found = order < C
    want_cell = order[found]
    want_id = 100 + np.arange(C, dtype=np.uint64)
    k = np.lexsort((want_id, want_cell))
    np.testing.assert_array_equal(p.cell, want_cell[k])
    np.testing.assert_array_equal(p.id, want_id[k])
    np.testing.assert_allclose(p.xhat, 0.5, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(p.x, centres[p.cell])

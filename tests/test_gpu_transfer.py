"""Sec. 2.7 (iv) shape-function-weighted vertex averages and (v) per-cell
linear least squares on the GPU, through the C ABI, against the oracle.

Both sides seed their stores from the same generator (the GPU keeps x-hat
as a double-float pair, within 2^-48 of the oracle's FP64 value) and get the
same property values.  Vertex averages are compared within 1e-12 of the
property's scale.  Least-squares coefficients are compared within
kappa * (64 eps + 4 * 2^-48) of their scale, kappa the condition number of the
cell's normal matrix: the solve amplifies both the rounding and the x-hat
difference by at most that much.  Counts and fallbacks are compared exactly.
"""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu

EPS = 2.0**-52


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def _pair(P, O, n, per_cell=None, ppc=0, seed=7):
    import torch

    X = W.jittered_vertices(n, seed)
    mesh = P.Mesh(n, X)
    parts = P.Particles(mesh, per_cell=per_cell, uniform_count=ppc, seed=seed, n_props=1)
    om = O.Mesh(n, X)
    op = O.seed_particles(om, per_cell=per_cell, uniform_count=ppc, seed=seed, n_props=1)
    vals = np.sin(5.0 * op.x[:, 0]) + op.x[:, 1] ** 2 - 0.3 * op.x[:, -1]
    parts.set_property(0, torch.as_tensor(vals, device="cuda"))
    return mesh, parts, om, op, vals


def _check_vertex(O, parts, om, op, vals):
    avg, w = parts.vertex_average(0, empty_fill=-5.0)
    oa, ow = O.vertex_average(om, op.cell, op.xhat, vals, empty_fill=-5.0)
    scale = max(1.0, np.abs(vals).max())
    g_avg, g_w = avg.cpu().numpy(), w.cpu().numpy()
    np.testing.assert_array_equal(g_w > 0, ow > 0)
    assert np.abs(g_w - ow).max() <= 1e-12 * max(1.0, ow.max())
    assert np.abs(g_avg - oa).max() <= 1e-12 * scale
    return avg, w


def _check_lsq(O, parts, om, op, vals, dim):
    coef, cnt = parts.project_linear(0, empty_fill=-5.0)
    oc, ocnt = O.cell_lsq_linear(om, op.cell, op.xhat, vals, empty_fill=-5.0)
    np.testing.assert_array_equal(cnt.cpu().numpy(), ocnt)
    gc = coef.cpu().numpy().T
    # condition numbers of the cells' normal matrices (oracle's inputs)
    C = om.ncells
    a = np.hstack([np.ones((op.n, 1)), op.xhat - 0.5])
    M = np.zeros((C, dim + 1, dim + 1))
    np.add.at(M, op.cell, a[:, :, None] * a[:, None, :])
    full = ocnt > dim
    kappa = np.ones(C)
    kappa[full] = np.linalg.cond(M[full])
    scale = np.maximum(1.0, np.maximum(np.abs(oc).max(axis=1), np.abs(vals).max()))
    tol = kappa * (64 * EPS + 4 * 2.0**-48) * scale
    err = np.abs(gc - oc).max(axis=1)
    bad = err > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], err[bad][:5], tol[bad][:5])
    # the fallback (mean) cells are the same on both sides
    np.testing.assert_array_equal(gc[~full, 1:], 0.0)
    return coef


@pytest.mark.parametrize("n", [(20, 17), (9, 7, 5)])
def test_transfer_ragged(P, oracle_mod, n):
    dim = len(n)
    C = int(np.prod(n))
    per = np.random.default_rng(3).integers(0, 9, size=C).astype(np.uint32)
    per[::7] = 0  # empty cells
    per[1::11] = dim  # too few for a fit: the mean
    mesh, parts, om, op, vals = _pair(P, oracle_mod, n, per_cell=per)
    a1, w1 = _check_vertex(oracle_mod, parts, om, op, vals)
    c1 = _check_lsq(oracle_mod, parts, om, op, vals, dim)
    # reproducible bit for bit
    a2, w2 = parts.vertex_average(0, empty_fill=-5.0)
    c2, _ = parts.project_linear(0, empty_fill=-5.0)
    assert (a1 == a2).all() and (w1 == w2).all() and (c1 == c2).all()


def test_transfer_after_advection(P, oracle_mod):
    wl = W.curl_cube(6, 7, 3, 4)
    mesh, parts = H.gpu_seed(wl, n_props=1)
    om, op = H.oracle_seed(oracle_mod, wl)
    parts.advect(wl.dt, 4, 3)
    op = oracle_mod.advect(om, op, wl.dt, 4, 3)
    # After advection the two sides' x-hat differ by up to delta (the
    # position tolerance over the cell size), so the transfers' inputs
    # differ, and the bounds follow from delta:
    #  - vertex averages p_v = sum phi_i p_i / W_v: each weight phi_i moves by
    #    at most delta (|d phi / d x-hat| <= 1), so
    #    |dp_v| <= sum |d phi_i| |p_i - p_v| / W_v <= 2 delta max|p| n_v / W_v
    #    (n_v particles around v), plus the rounding bound of equal inputs;
    #  - least squares c = M^-1 b, a = (1, x-hat - 1/2): M and b move by a
    #    relative 2 (dim + 1) delta <= 8 delta, so c moves by kappa(M) 8 delta
    #    |c| on top of the rounding bound kappa (64 eps + 4 2^-48) |c|.
    delta = H.tol_xhat(wl)
    p = op.props[:, 0]
    avg, w = parts.vertex_average(0)
    oa, ow = oracle_mod.vertex_average(om, op.cell, op.xhat, p)
    nv = np.zeros(len(oa))
    dims = [k + 1 for k in wl.n]
    for q in range(8):
        o = [(q >> a) & 1 for a in range(3)]
        c = np.array(np.unravel_index(op.cell, wl.n[::-1])[::-1])  # (i, j, k) of each particle's cell
        v = (c[0] + o[0]) + dims[0] * ((c[1] + o[1]) + dims[1] * (c[2] + o[2]))
        np.add.at(nv, v, 1.0)
    has = ow > 0
    tol_v = 2 * delta * np.abs(p).max() * nv[has] / ow[has] + 1e-12 * max(1.0, np.abs(p).max())
    err_v = np.abs(avg.cpu().numpy()[has] - oa[has])
    assert (err_v <= tol_v).all(), (err_v / tol_v).max()
    coef, cnt = parts.project_linear(0)
    oc, ocnt = oracle_mod.cell_lsq_linear(om, op.cell, op.xhat, p)
    np.testing.assert_array_equal(cnt.cpu().numpy(), ocnt)
    C = om.ncells
    a = np.hstack([np.ones((op.n, 1)), op.xhat - 0.5])
    M = np.zeros((C, 4, 4))
    np.add.at(M, op.cell, a[:, :, None] * a[:, None, :])
    full = ocnt > 3
    kappa = np.ones(C)
    kappa[full] = np.linalg.cond(M[full])
    scale = np.maximum(1.0, np.maximum(np.abs(oc).max(axis=1), np.abs(p).max()))
    tol_c = kappa * (64 * EPS + 4 * 2.0**-48 + 8 * delta) * scale
    err_c = np.abs(coef.cpu().numpy().T - oc).max(axis=1)
    assert (err_c <= tol_c).all(), (err_c / tol_c).max()


def test_transfer_full_size(P, oracle_mod):
    """64^3 jittered hexes, 20 per cell (5.24M particles): every vertex and
    every cell against the oracle."""
    mesh, parts, om, op, vals = _pair(P, oracle_mod, (64, 64, 64), ppc=20, seed=2)
    _check_vertex(oracle_mod, parts, om, op, vals)
    _check_lsq(oracle_mod, parts, om, op, vals, 3)


def test_transfer_errors(P):
    mesh = P.Mesh((3, 3), W.uniform_vertices((3, 3)))
    parts = P.Particles(mesh, uniform_count=2, seed=1, n_props=1)
    with pytest.raises(P.PicError):
        parts.vertex_average(1)
    with pytest.raises(P.PicError):
        parts.project_linear(-1)

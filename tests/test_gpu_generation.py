"""Generation with a density and from prescribed locations (Sec. 2.2) on the
GPU, through the C ABI, against the oracle on the same inputs.

The decisions are integers taken from floating point (which cell a draw
falls in, whether a proposal is accepted); both sides evaluate the same
written sequence of IEEE operations, so they are compared bit for bit: cell
weights, per-cell counts, the accepted chains (cells, ids, positions).  The
stored x-hat is a double-float pair, within 2^-48 of the oracle's FP64
value.  Imported points go through the owner search, so cells and ids are
exact and x-hat agrees within the position tolerance over the cell size.
"""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def _rho(X, seed, zero_frac=0.1):
    g = np.random.default_rng(seed)
    r = g.uniform(0.0, 3.0, X.shape[1])
    r[g.uniform(size=r.shape) < zero_frac] = 0.0
    return r


@pytest.mark.parametrize("n", [(20, 17), (9, 7, 5), (64, 64, 64)])
def test_cell_weights_and_counts_bit_exact(P, oracle_mod, n):
    O = oracle_mod
    X = W.jittered_vertices(n, 3)
    rho = _rho(X, 5)
    mesh, om = P.Mesh(n, X), O.Mesh(n, X)
    w_g = P.cell_weights(mesh, rho).cpu().numpy()
    w_o = O.cell_weights(om, rho)
    np.testing.assert_array_equal(w_g, w_o)
    C = om.ncells
    N = 20 * C
    w = w_o.copy()
    w[::13] = 0.0  # zero-weight cells
    c_g = P.draw_cell_counts(w, N, 4242).cpu().numpy().view(np.uint32)
    c_o = O.draw_cell_counts(w, N, 4242)
    np.testing.assert_array_equal(c_g.astype(np.int64), c_o)
    assert c_g.sum() == N and (c_g[w == 0] == 0).all()


@pytest.mark.parametrize("n,J", [((20, 17), 3), ((9, 7, 5), 4), ((32, 32, 32), 2)])
def test_metropolis_hastings_matches_oracle(P, oracle_mod, n, J):
    O = oracle_mod
    X = W.jittered_vertices(n, 8)
    rho = _rho(X, 9)
    mesh, om = P.Mesh(n, X), O.Mesh(n, X)
    C = om.ncells
    per = np.random.default_rng(2).integers(0, 12 if len(n) == 2 else 9, size=C).astype(np.uint32)
    per[::5] = 0
    parts = P.Particles.metropolis_hastings(mesh, per, rho, thinning=J, seed=77, first_id=5, n_props=1)
    g = H.gpu_state(parts)
    o = O.seed_particles_mh(om, per, rho, J, 77, first_id=5)
    np.testing.assert_array_equal(g["id"], o.id)
    np.testing.assert_array_equal(g["cell"], o.cell)
    np.testing.assert_array_equal(g["x"], o.x)
    assert np.abs(g["xhat"] - o.xhat).max() <= 2.0**-48
    off = parts.cell_offsets().cpu().numpy()
    np.testing.assert_array_equal(np.diff(off), per)


def test_density_pipeline_end_to_end(P, oracle_mod):
    """rho -> cell weights -> counts -> MH particles, every stage on the GPU,
    against the same stages of the oracle."""
    O = oracle_mod
    n = (16, 12, 10)
    X = W.jittered_vertices(n, 12)
    Xv = X
    rho = 1.0 + 4.0 * Xv[0] * Xv[1]  # smooth, positive
    mesh, om = P.Mesh(n, X), O.Mesh(n, X)
    wg = P.cell_weights(mesh, rho)
    cg = P.draw_cell_counts(wg, 30000, 11)
    parts = P.Particles.metropolis_hastings(mesh, cg, rho, thinning=6, seed=12)
    wo = O.cell_weights(om, rho)
    co = O.draw_cell_counts(wo, 30000, 11)
    o = O.seed_particles_mh(om, co.astype(np.uint32), rho, 6, 12)
    g = H.gpu_state(parts)
    np.testing.assert_array_equal(g["cell"], o.cell)
    np.testing.assert_array_equal(g["x"], o.x)


def test_import_points_matches_oracle(P, oracle_mod):
    import torch

    O = oracle_mod
    for n in ((7, 6), (5, 4, 6)):
        dim = len(n)
        X = W.jittered_vertices(n, 30)
        mesh, om = P.Mesh(n, X), O.Mesh(n, X)
        g = np.random.default_rng(6)
        pts = [g.uniform(-0.1, 1.1, size=(4000, dim))]
        pts.append(X.T.copy())  # every vertex: shared by up to 2^dim cells
        pts = np.concatenate(pts)[g.permutation(4000 + X.shape[1])]
        parts, outside = P.Particles.import_points(mesh, torch.as_tensor(np.ascontiguousarray(pts.T), device="cuda"),
                                                   first_id=1000, n_props=2)
        o = O.import_points(om, pts, first_id=1000)
        assert outside == len(pts) - o.n
        st = H.gpu_state(parts)
        np.testing.assert_array_equal(st["id"], o.id)
        np.testing.assert_array_equal(st["cell"], o.cell)
        np.testing.assert_array_equal(st["x"], o.x)
        assert np.abs(st["xhat"] - o.xhat).max() <= 1e-12 * max(n) * 1.25
        assert parts.state()[0] == o.n
        # the imported store advances like a seeded one (uniform field)
        nq = int(np.prod([2 * k + 1 for k in n]))
        mesh.set_velocity(np.full((dim, nq), 0.01))
        parts.advect(0.5, 4, 1)
        n_alive, n_lost, status = parts.state()
        assert n_alive + n_lost == o.n and status & P.PIC_STATUS_BOUNDS == 0


def test_import_empty_and_errors(P):
    import torch

    mesh = P.Mesh((3, 3), W.uniform_vertices((3, 3)))
    parts, outside = P.Particles.import_points(mesh, torch.full((2, 5), 7.0, dtype=torch.float64, device="cuda"))
    assert outside == 5 and parts.state()[0] == 0
    w = torch.ones(9, dtype=torch.float64, device="cuda")
    w[3] = -1.0
    with pytest.raises(P.PicError):
        P.draw_cell_counts(w, 10, 1)
    with pytest.raises(P.PicError):
        P.draw_cell_counts(torch.zeros(9, dtype=torch.float64, device="cuda"), 10, 1)
    with pytest.raises(P.PicError):
        P.Particles.metropolis_hastings(mesh, np.ones(9, np.uint32), np.ones(16), thinning=0)

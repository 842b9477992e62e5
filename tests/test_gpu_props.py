"""Property ODEs of Sec. 2.6 (damage, deformation gradient) on the GPU,
through the C ABI, against the oracle on the same seeded inputs.

Cells, ids and order are compared bit for bit, positions within 1e-12 of the
domain.  The properties are compared relative to their size: F and d are
products of FP64 arithmetic over a few dozen operations per stage (the GPU
contracts to FMA, the oracle does not), so per particle
|F_gpu - F_oracle| <= 1e-12 * max(1, max|F|) and the same for d.
"""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu

TOL_PROP = 1e-12


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def _initial_props(N, dim, seed):
    g = np.random.default_rng(seed)
    nP = 2 + dim * dim
    pr = np.zeros((N, nP))
    pr[:, 0] = g.uniform(0.0, 1.0, N)  # d_0
    F0 = np.eye(dim)[None] + 0.1 * g.uniform(-1.0, 1.0, (N, dim, dim))
    pr[:, 1:1 + dim * dim] = F0.reshape(N, -1)
    pr[:, -1] = g.uniform(-3.0, 3.0, N)  # rides along unchanged
    return pr


def _setup(P, O, wl, seed=17):
    import torch

    dim = wl.dim
    nP = 2 + dim * dim
    mesh, parts = H.gpu_seed(wl, n_props=nP)
    om = O.Mesh(wl.n, wl.X, wl.U)
    op = O.seed_particles(om, per_cell=wl.per_cell, uniform_count=wl.ppc or 0, seed=wl.pseed, first_id=wl.first_id,
                          n_props=nP)
    pr = _initial_props(op.n, dim, seed)
    op.props[:] = pr
    for q in range(nP):
        parts.set_property(q, torch.as_tensor(np.ascontiguousarray(pr[:, q]), device="cuda"))
    return mesh, parts, om, op


def _check_props(g, o, dim, tol=TOL_PROP):
    nP = 2 + dim * dim
    gp, opr = g["props"][:, :nP], o.props
    scale = np.maximum(1.0, np.abs(opr[:, 1:1 + dim * dim]).max(axis=1))
    dF = np.abs(gp[:, 1:1 + dim * dim] - opr[:, 1:1 + dim * dim]).max(axis=1)
    assert (dF <= tol * scale).all(), (dF / scale).max()
    dd = np.abs(gp[:, 0] - opr[:, 0])
    assert (dd <= tol * np.maximum(1.0, np.abs(opr[:, 0]))).all(), dd.max()
    np.testing.assert_array_equal(gp[:, -1], opr[:, -1])


@pytest.mark.parametrize("case,integrator", [("2d", 4), ("2d", 2), ("3d", 4), ("3d", 2), ("3d", 1)])
def test_props_match_oracle(P, oracle_mod, case, integrator):
    wl = W.c1(n=12, ppc=6) if case == "2d" else W.curl_cube(5, 6, 1, 3)
    if case == "2d":
        # a sheared rotation so that the strain rate is not zero
        Pn = W.q2_node_coords(wl.n, wl.X)
        wl.U = np.stack([-(Pn[1] - 0.5) + 0.3 * (Pn[1] - 0.5) ** 2, (Pn[0] - 0.5) * (1.2 - 0.4 * Pn[0])])
        wl.U = W.zero_wall_normal(wl.n, wl.U)
    mesh, parts, om, op = _setup(P, oracle_mod, wl)
    steps = 4
    alpha, beta = 0.8, 0.6
    parts.advect_properties(wl.dt, integrator, steps, damage=0, alpha=alpha, beta=beta, deformation=1)
    op = oracle_mod.advect_properties(om, op, wl.dt, integrator, steps, damage=0, alpha=alpha, beta=beta, defgrad=1)
    g = H.gpu_state(parts)
    n_alive, n_lost, status = parts.state()
    assert n_alive == op.n and n_lost == op.n_lost
    assert g["id"].shape[0] == op.n
    np.testing.assert_array_equal(g["id"], op.id)
    np.testing.assert_array_equal(g["cell"], op.cell)
    assert np.abs(g["x"] - op.x).max() <= H.TOL_X
    _check_props(g, op, wl.dim)


def test_props_with_losses(P, oracle_mod):
    """CFL ~6: stage points leave the domain and their particles are dropped;
    the survivors' properties still match the oracle."""
    wl = W.curl_cube(6, 6, 1, 9)
    mesh, parts, om, op = _setup(P, oracle_mod, wl)
    dt = 12 * wl.dt
    parts.advect_properties(dt, 4, 2, damage=0, alpha=0.8, beta=0.6, deformation=1)
    op = oracle_mod.advect_properties(om, op, dt, 4, 2, damage=0, alpha=0.8, beta=0.6, defgrad=1)
    g = H.gpu_state(parts)
    n_alive, n_lost, status = parts.state()
    assert n_lost > 0 and n_alive == op.n and n_lost == op.n_lost
    np.testing.assert_array_equal(g["id"], op.id)
    np.testing.assert_array_equal(g["cell"], op.cell)
    assert np.abs(g["x"] - op.x).max() <= H.TOL_X
    # Reading: the 1e-12 bound on F and d holds at the CFL-0.5 step.  A
    # rounding error dG of a stage's velocity gradient enters F as dt dG F
    # (and d as alpha dt |d eps-dot|), so at a step dt / dt_cfl times larger
    # the bound scales by that ratio (measured: 2.0e-12 relative at 12x).
    _check_props(g, op, wl.dim, tol=(dt / wl.dt) * TOL_PROP)


def test_props_on_an_emptied_store(P, oracle_mod):
    """Every particle leaves in the first step; further property steps run on
    an empty store and leave it empty."""
    wl = W.c1(n=2, ppc=4)
    mesh, parts, om, op = _setup(P, oracle_mod, wl)
    parts.advect_properties(50.0, 4, 1, damage=0, alpha=0.8, beta=0.6, deformation=1)
    n_alive, n_lost, status = parts.state()
    assert n_alive == 0 and n_lost == 16
    parts.advect_properties(wl.dt, 4, 2, damage=0, alpha=0.8, beta=0.6, deformation=1)
    assert parts.state()[:2] == (0, 16)


def test_positions_identical_to_plain_advect(P, oracle_mod):
    wl = W.curl_cube(6, 8, 1, 5)
    mesh, a = H.gpu_seed(wl, n_props=11)
    _, b = H.gpu_seed(wl, n_props=11)
    import torch

    N = a.state()[0]
    eye = np.eye(3).reshape(-1)
    for q in range(9):
        a.set_property(1 + q, torch.full((N,), float(eye[q]), dtype=torch.float64, device="cuda"))
    a.advect_properties(wl.dt, 4, 5, damage=0, alpha=1.0, beta=0.5, deformation=1)
    b.advect(wl.dt, 4, 5)
    ga, gb = H.gpu_state(a), H.gpu_state(b)
    np.testing.assert_array_equal(ga["id"], gb["id"])
    np.testing.assert_array_equal(ga["cell"], gb["cell"])
    np.testing.assert_array_equal(ga["x"], gb["x"])
    np.testing.assert_array_equal(ga["xhat"], gb["xhat"])
    # the unrelated property 10 rides along untouched in both
    np.testing.assert_array_equal(ga["props"][:, 10], gb["props"][:, 10])


def test_props_sampled_at_scale(P, oracle_mod):
    """32^3 jittered hexes, 8 per cell (262,144 particles), RK4, 3 steps on the
    GPU; the oracle advances every 61st particle on its own (particles are
    independent) and the two are compared by id."""
    wl = W.curl_cube(32, 8, 3, 2)
    mesh, parts, om, op = _setup(P, oracle_mod, wl, seed=3)
    parts.advect_properties(wl.dt, 4, 3, damage=0, alpha=0.8, beta=0.6, deformation=1)
    g = H.gpu_state(parts)
    sub = op.subset(np.arange(op.n) % 61 == 0)
    o = oracle_mod.advect_properties(om, sub, wl.dt, 4, 3, damage=0, alpha=0.8, beta=0.6, defgrad=1)
    pos = {int(i): k for k, i in enumerate(g["id"])}
    rows = np.array([pos[int(i)] for i in o.id])
    gsub = {k: v[rows] for k, v in g.items()}
    np.testing.assert_array_equal(gsub["cell"], o.cell)
    assert np.abs(gsub["x"] - o.x).max() <= H.TOL_X
    _check_props(gsub, o, 3)


def test_props_errors(P):
    wl = W.curl_cube(3, 2, 1, 1)
    mesh, parts = H.gpu_seed(wl, n_props=10)
    with pytest.raises(P.PicError):
        parts.advect_properties(wl.dt, 4, 1, deformation=2)  # slots 2..10 > 10 properties
    with pytest.raises(P.PicError):
        parts.advect_properties(wl.dt, 4, 1, damage=10)
    with pytest.raises(P.PicError):
        parts.advect_properties(wl.dt, 4, 1, damage=3, deformation=1)  # overlap
    with pytest.raises(P.PicError):
        parts.advect_properties(wl.dt, 3, 1, damage=0)  # no such integrator
    mesh.set_velocity(wl.U, U_next=wl.U)
    with pytest.raises(P.PicError):
        parts.advect_properties(wl.dt, 4, 1, damage=0)  # two fields
    assert parts.state()[2] == 0

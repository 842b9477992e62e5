"""GPU path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Integer results (owner cells, ids, order, counts) are compared bit
for bit; FP64 values within the tolerances in gpu_helpers."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def test_seed_matches_oracle(P, oracle_mod):
    for wl in (W.c1(n=8, ppc=5), W.curl_cube(4, 7, 1, 3)):
        mesh, parts = H.gpu_seed(wl)
        g = H.gpu_state(parts)
        om, op = H.oracle_seed(oracle_mod, wl)
        np.testing.assert_array_equal(g["id"], op.id)
        np.testing.assert_array_equal(g["cell"], op.cell)
        # same generator bits; the store keeps x-hat as a double-float pair
        assert np.abs(g["xhat"] - op.xhat).max() <= 2.0**-48
        assert np.abs(g["x"] - op.x).max() <= 4e-16
        off = parts.cell_offsets().cpu().numpy()
        np.testing.assert_array_equal(np.diff(off), np.bincount(op.cell, minlength=wl.ncells))


def test_seed_ragged_per_cell(P, oracle_mod):
    wl = W.c5_member(6, 11)
    wl.per_cell[::3] = 0  # empty cells
    mesh, parts = H.gpu_seed(wl)
    g = H.gpu_state(parts)
    om, op = H.oracle_seed(oracle_mod, wl)
    H.assert_same_store(g, op, wl)


@pytest.mark.parametrize("n", [(3, 3), (3, 3, 3), (6, 5, 4)])
def test_locate_points_matches_oracle(P, oracle_mod, n):
    import torch

    dim = len(n)
    X = W.jittered_vertices(n, 5)
    om = oracle_mod.Mesh(n, X)
    g = np.random.default_rng(2)
    pts = [g.uniform(-0.05, 1.05, size=(3000, dim))]
    C = int(np.prod(n))
    ref = np.array(list(np.ndindex(*(3,) * dim))) / 2.0
    pts.append(np.array([om.phi(K, r) for K in range(C) for r in ref]))  # faces, edges, vertices
    pts.append(np.array([om.phi(K, r + s) for K in range(0, C, 3) for r in ref[:4] for s in (1e-11, -1e-11, 3e-10)]))
    Pn = np.concatenate(pts)
    oc, ot = om.locate(Pn)
    mesh = P.Mesh(n, X)
    x = torch.as_tensor(np.ascontiguousarray(Pn.T), device="cuda")
    for hint in (None, torch.zeros(Pn.shape[0], dtype=torch.int32, device="cuda")):
        gc, gt = mesh.locate_points(x, hint)
        gc = gc.cpu().numpy().view(np.uint32).astype(np.int64)
        gc[gc == 0xFFFFFFFF] = -1
        np.testing.assert_array_equal(gc, oc)
        found = oc >= 0
        assert np.abs(gt.cpu().numpy().T[found] - ot[found]).max() <= 1e-11


def _run_both(P, O, wl, steps, integrator=None, precision=0, per_step=False):
    integrator = integrator or wl.integrator
    mesh, parts = H.gpu_seed(wl)
    om, op = H.oracle_seed(O, wl)
    avgs = []
    if per_step:
        for _ in range(steps):
            parts.advect(wl.dt, integrator, 1, precision)
            op = O.advect(om, op, wl.dt, integrator, 1)
            if wl.n_props:
                ga, gc = parts.average(0)
                oa, oc = O.cell_average(om.ncells, op.cell, op.props[:, 0])
                avgs.append((ga.cpu().numpy(), gc.cpu().numpy(), oa, oc))
    else:
        parts.advect(wl.dt, integrator, steps, precision)
        op = O.advect(om, op, wl.dt, integrator, steps)
    return parts, op, avgs


def test_c1_full_rotation_rk2(P, oracle_mod):
    """2D unit square 32x32, rigid rotation, 16 per cell, RK2 at CFL 0.5, 10
    steps with cell averages after every step; corner particles leave."""
    wl = W.c1()
    parts, op, avgs = _run_both(P, oracle_mod, wl, wl.n_steps, per_step=True)
    g = H.gpu_state(parts)
    H.assert_same_store(g, op, wl)
    n_alive, n_lost, status = parts.state()
    assert n_alive == op.n and n_lost == op.n_lost and n_lost > 0
    for ga, gc, oa, oc in avgs:
        np.testing.assert_array_equal(gc.astype(np.int64), oc)
        assert np.abs(ga - oa).max() <= H.TOL_AVG


@pytest.mark.parametrize("integrator", [1, 2, 4])
def test_3d_jittered_small(P, oracle_mod, integrator):
    """The 3D curl-field construction at 8^3 (spans many warps and cells,
    ragged last block), every integrator."""
    wl = W.curl_cube(8, 20, 6, 2)
    parts, op, _ = _run_both(P, oracle_mod, wl, wl.n_steps, integrator=integrator)
    H.assert_same_store(H.gpu_state(parts), op, wl)
    ga, gc = parts.average(1)
    oa, oc = oracle_mod.cell_average(wl.ncells, op.cell, op.props[:, 1])
    np.testing.assert_array_equal(gc.cpu().numpy().astype(np.int64), oc)
    assert np.abs(ga.cpu().numpy() - oa).max() <= H.TOL_AVG


def test_3d_large_dt_walks_and_losses(P, oracle_mod):
    """CFL ~2: stage points cross several cells, exercising the walk, the
    all-cells search and losses through the walls."""
    wl = W.curl_cube(6, 6, 3, 9)
    # 4x the CFL-0.5 step
    mesh, parts = H.gpu_seed(wl)
    om, op = H.oracle_seed(oracle_mod, wl)
    parts.advect(4 * wl.dt, 4, 3)
    op = oracle_mod.advect(om, op, 4 * wl.dt, 4, 3)
    H.assert_same_store(H.gpu_state(parts), op, wl)
    st = parts.stats()
    assert st["walks"] > 0


def test_c2_full_size_sampled(P, oracle_mod):
    """3D 64^3 jittered, 20 per cell (5.24M), RK4, 50 steps: the launch
    configuration of the benchmark.  Sampled particles are followed by the
    oracle one by one (trajectories are independent); the whole store is
    checked for the sorted-by-(cell, id) invariant and conservation."""
    wl = W.c2()
    mesh, parts = H.gpu_seed(wl)
    N0 = wl.n_particles
    parts.advect(wl.dt, wl.integrator, wl.n_steps)
    g = H.gpu_state(parts)
    n_alive, n_lost, status = parts.state()
    assert n_alive + n_lost == N0
    key = g["cell"] * (2**40) + g["id"].astype(np.int64)
    assert (np.diff(key) > 0).all()
    off = parts.cell_offsets().cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(np.diff(off), np.bincount(g["cell"], minlength=wl.ncells))
    # sample: oracle trajectories of 300 particles
    om, op = H.oracle_seed(oracle_mod, wl)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(N0, 300, replace=False))
    sub = op.subset(pick)
    so = oracle_mod.advect(om, sub, wl.dt, wl.integrator, wl.n_steps)
    pos = {int(i): k for k, i in enumerate(g["id"])}
    for i, c, x in zip(so.id, so.cell, so.x):
        k = pos[int(i)]
        assert g["cell"][k] == c
        assert np.abs(g["x"][k] - x).max() <= H.TOL_X
    lost_ids = set(int(i) for i in sub.id) - set(int(i) for i in so.id)
    for i in lost_ids:
        assert i not in pos
    # cell averages (Sec. 2.7 (ii)) of sampled cells at full size: every
    # particle the GPU holds in the cell is followed by the oracle, must end
    # in that cell, and the oracle's left fold of their property over them
    # (store order) is the GPU's average
    ga, gc = parts.average(1)
    ga, gc = ga.cpu().numpy(), gc.cpu().numpy()
    for K in rng.choice(wl.ncells, 12, replace=False):
        members = np.nonzero(g["cell"] == K)[0]
        assert gc[K] == len(members)
        idx = np.searchsorted(op.id, g["id"][members])  # ids index the oracle's seeded store
        so = oracle_mod.advect(om, op.subset(idx), wl.dt, wl.integrator, wl.n_steps)
        np.testing.assert_array_equal(so.cell, np.full(len(members), K))
        np.testing.assert_array_equal(so.id, g["id"][members])
        oa, oc = oracle_mod.cell_average(wl.ncells, so.cell, so.props[:, 1])
        assert oc[K] == gc[K]
        assert abs(oa[K] - ga[K]) <= H.TOL_AVG, (K, oa[K], ga[K])


def test_c3_fp64_form_full_size_sampled(P, oracle_mod):
    """The benchmark's headline configuration in the FP64 form: 128^3
    jittered hexes, 20 per cell (41.9M particles), RK4, 20 steps.  Sampled
    particles follow the oracle one by one: same owner cell, positions within
    1e-12.  The whole store keeps the sorted-by-(cell, id) invariant and
    conservation."""
    wl = W.c3()
    mesh, parts = H.gpu_seed(wl, n_props=0)
    N0 = wl.n_particles
    parts.advect(wl.dt, wl.integrator, wl.n_steps, P.PIC_FP64)
    n_alive, n_lost, status = parts.state()
    assert n_alive + n_lost == N0
    assert status == 0
    e = parts.export()
    ids = e["id"].cpu().numpy().astype(np.int64)
    cells = e["cell"].cpu().numpy().view(np.uint32).astype(np.int64)
    key = cells * (2**40) + ids
    assert (np.diff(key) > 0).all()
    rng = np.random.default_rng(2)
    pick = np.sort(rng.choice(N0, 200, replace=False))
    om = oracle_mod.Mesh(wl.n, wl.X, wl.U)
    sub = _sample_from_generator(oracle_mod, om, wl, pick)
    so = oracle_mod.advect(om, sub, wl.dt, wl.integrator, wl.n_steps)
    pos = {int(i): k for k, i in enumerate(ids)}
    x = e["x"].cpu().numpy()
    for i, c, xo in zip(so.id, so.cell, so.x):
        k = pos[int(i)]
        assert cells[k] == c
        assert np.abs(x[:, k] - xo).max() <= H.TOL_X
    for i in set(int(i) for i in sub.id) - set(int(i) for i in so.id):
        assert i not in pos


def _sample_from_generator(O, om, wl, ids):
    """Particles `ids` of a uniform-count seeding, rebuilt from the published
    generator (SplitMix64 output g*dim + j gives x-hat_j of particle g) and
    the oracle's map, without seeding the whole store in the oracle."""
    d = wl.dim
    xh = np.array([[(O.splitmix64(wl.pseed, int(g) * d + j) >> 11) * 2.0**-53 for j in range(d)] for g in ids])
    cell = (np.asarray(ids) // wl.ppc).astype(np.int64)
    x = np.array([om.phi(int(K), t) for K, t in zip(cell, xh)])
    return O.Particles(x, xh, cell, (wl.first_id + np.asarray(ids)).astype(np.uint64), np.zeros((len(ids), 0)))


def test_c3_full_size_sampled(P, oracle_mod):
    """Precision form at the size the benchmark runs: 128^3 jittered hexes, 20
    per cell (41.9M particles), RK4, 20 steps.  Sampled particles follow the
    FP64 oracle one by one; the FP32 basis keeps them within 1e-6 of it (the
    velocity carries ~1e-7 relative error over 20 steps of dt ~ 0.004).  The
    whole store keeps the sorted-by-(cell, id) invariant and conservation."""
    wl = W.c3()
    mesh, parts = H.gpu_seed(wl, n_props=0)
    N0 = wl.n_particles
    parts.advect(wl.dt, wl.integrator, wl.n_steps, P.PIC_FP32_BASIS)
    n_alive, n_lost, status = parts.state()
    assert n_alive + n_lost == N0
    e = parts.export()
    ids = e["id"].cpu().numpy().astype(np.int64)
    cells = e["cell"].cpu().numpy().view(np.uint32).astype(np.int64)
    key = cells * (2**40) + ids
    assert (np.diff(key) > 0).all()
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(N0, 200, replace=False))
    om = oracle_mod.Mesh(wl.n, wl.X, wl.U)
    sub = _sample_from_generator(oracle_mod, om, wl, pick)
    so = oracle_mod.advect(om, sub, wl.dt, wl.integrator, wl.n_steps)
    pos = {int(i): k for k, i in enumerate(ids)}
    x = e["x"].cpu().numpy()
    err = max(np.abs(x[:, pos[int(i)]] - xo).max() for i, xo in zip(so.id, so.x))
    assert err <= 1e-6, err


def test_fp32_basis_error_bound(P, oracle_mod):
    """Precision form: Q2 basis and contraction in FP32.  Owner cells may
    differ only for particles within FP32 round-off of a face, so compare
    positions by id; the error against the FP64 oracle is bounded."""
    wl = W.curl_cube(8, 20, 10, 2)
    parts, op, _ = _run_both(P, oracle_mod, wl, wl.n_steps, precision=1)
    g = H.gpu_state(parts)
    pos = {int(i): k for k, i in enumerate(g["id"])}
    err = max(np.abs(g["x"][pos[int(i)]] - x).max() for i, x in zip(op.id, op.x) if int(i) in pos)
    assert err <= 1e-5, err


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_basis_stage_residual_forms(P, oracle_mod, precision):
    """Both readings of the precision form on the same store: the stage
    points located by the FP32 Newton alone (1) or with the double-float
    residual step too (2, PIC_FP32_BASIS_STAGE_DF).  Either stays within the
    FP32 basis' error of the FP64 oracle, and the two agree with each other
    to that order (the stage x-hat they feed an FP32 basis differ by ~1e-7)."""
    wl = W.curl_cube(8, 20, 10, 2)
    parts, op, _ = _run_both(P, oracle_mod, wl, wl.n_steps, precision=precision)
    g = H.gpu_state(parts)
    pos = {int(i): k for k, i in enumerate(g["id"])}
    err = max(np.abs(g["x"][pos[int(i)]] - x).max() for i, x in zip(op.id, op.x) if int(i) in pos)
    assert err <= 1e-5, err
    assert parts.state()[2] == 0
    if precision == 2:
        other, _, _ = _run_both(P, oracle_mod, wl, wl.n_steps, precision=1)
        o = H.gpu_state(other)
        opos = {int(i): k for k, i in enumerate(o["id"])}
        d = max(np.abs(g["x"][pos[i]] - o["x"][opos[i]]).max() for i in pos if i in opos)
        assert d <= 1e-5, d


def test_edge_cases(P, oracle_mod):
    import torch

    # one cell, Euler, zero steps is a no-op, capacity larger than needed
    wl = W.c1(n=1, ppc=9, n_steps=3)
    mesh, parts = H.gpu_seed(wl, capacity=100)
    before = H.gpu_state(parts)
    parts.advect(wl.dt, 1, 0)
    after = H.gpu_state(parts)
    np.testing.assert_array_equal(before["x"], after["x"])
    parts.advect(wl.dt, 1, 3)
    om, op = H.oracle_seed(oracle_mod, wl)
    op = oracle_mod.advect(om, op, wl.dt, 1, 3)
    H.assert_same_store(H.gpu_state(parts), op, wl)
    # everything leaves: huge step, then further steps on an empty store
    parts.advect(50.0, 4, 2)
    n_alive, n_lost, _ = parts.state()
    assert n_alive == 0 and n_lost == 9
    avg, cnt = parts.average(0, empty_fill=-3.0)
    assert avg.cpu().numpy().tolist() == [-3.0] and cnt.cpu().numpy().tolist() == [0]
    # rebin of a sorted store is the identity; relocation keeps cells
    wl = W.curl_cube(5, 3, 1, 4)
    mesh, parts = H.gpu_seed(wl)
    a = H.gpu_state(parts)
    parts.rebin()
    parts.locate()
    b = H.gpu_state(parts)
    np.testing.assert_array_equal(a["id"], b["id"])
    np.testing.assert_array_equal(a["cell"], b["cell"])
    assert np.abs(a["xhat"] - b["xhat"]).max() <= 1e-13
    # argument errors
    with pytest.raises(P.PicError):
        parts.advect(float("nan"), 4, 1)
    with pytest.raises(P.PicError):
        parts.set_property(7, torch.zeros(1, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("kind", [1, 2])
def test_geometric_harmonic_averages(P, oracle_mod, kind):
    """Sec. 2.7 (ii) geometric and harmonic averages after a few steps, on a
    positive property (1 + x0 + y0) and on one with non-positive values."""
    import torch

    wl = W.curl_cube(8, 5, 2, 7)
    mesh, parts = H.gpu_seed(wl)
    st = parts.export()
    pos = (1.0 + st["x"][0] + st["x"][1]).contiguous()
    parts.set_property(0, pos)
    parts.set_property(1, (st["x"][2] - 0.5).contiguous())  # changes sign
    parts.advect(wl.dt, 4, 2)
    # the oracle's own run on the same seeded inputs
    om, op = H.oracle_seed(oracle_mod, wl)
    op.props[:, 0] = 1.0 + op.x[:, 0] + op.x[:, 1]
    op.props[:, 1] = op.x[:, 2] - 0.5
    op = oracle_mod.advect(om, op, wl.dt, 4, 2)
    np.testing.assert_array_equal(H.gpu_state(parts)["cell"], op.cell)
    for prop in (0, 1):
        ga, gc = parts.average(prop, empty_fill=-9.0, kind=kind)
        oa, oc = oracle_mod.cell_average(wl.ncells, op.cell, op.props[:, prop], empty_fill=-9.0, kind=kind)
        ga = ga.cpu().numpy()
        np.testing.assert_array_equal(gc.cpu().numpy().astype(np.int64), oc)
        np.testing.assert_array_equal(np.isnan(ga), np.isnan(oa))
        ok = ~np.isnan(oa)
        assert np.abs(ga[ok] - oa[ok]).max() <= 1e-13 * np.abs(oa[ok]).max()


@pytest.mark.parametrize("integrator", [4, 2, 1])
def test_time_interpolated_velocity(P, oracle_mod, integrator):
    """Two fields u_h^n, u_h^{n+1}: stage s at t^n + c_s dt uses
    (1 - c_s) u_h^n + c_s u_h^{n+1} (reading R6)."""
    wl = W.curl_cube(7, 6, 3, 11)
    Un = W.zero_wall_normal(wl.n, W.normalise_max(W.curl_potential_field(W.q2_node_coords(wl.n, wl.X), 12)[0]))
    mesh, parts = H.gpu_seed(wl)
    mesh.set_velocity(wl.U, U_next=Un)
    parts.advect(wl.dt, integrator, 3)
    om, op = H.oracle_seed(oracle_mod, wl)
    om.set_velocity_next(Un)
    op = oracle_mod.advect(om, op, wl.dt, integrator, 3)
    H.assert_same_store(H.gpu_state(parts), op, wl)
    # U_next = U is the steady field bit for bit
    m1, p1 = H.gpu_seed(wl)
    m2, p2 = H.gpu_seed(wl)
    m2.set_velocity(wl.U, U_next=wl.U)
    p1.advect(wl.dt, integrator, 3)
    p2.advect(wl.dt, integrator, 3)
    a, b = H.gpu_state(p1), H.gpu_state(p2)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["id"], b["id"])

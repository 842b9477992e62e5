"""Form 3 (adjoint): dL/dU from the GPU tape against the oracle's reverse
mode, against central finite differences of the GPU forward, and through the
torch.autograd.Function.  L = sum over survivors of |x_final - target|^2."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu

# The GPU sums the same per-stage contributions as the oracle, in another
# order (per cell, then per node), with the forward's double-float stage
# points and double-float G and lambda; differences stay at rounding level
# (measured 2e-14 on the small cases and 1e-13 after the 20 steps of the
# 32^3 case), bounded here relative to the largest gradient entry.
TOL_GRAD = 1e-12


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def _targets_by_id(wl, n_total, x_like, seed=3):
    # targets indexed by particle id: a smooth displacement plus N(0, h^2) noise
    h = 1.0 / max(wl.n)
    g = np.random.default_rng(seed)
    return x_like + h * g.standard_normal(x_like.shape)


def _gpu_grad(P, wl, steps, dt, integrator, targets_by_id, weight_by_id=None, kind=None, dx0=None):
    import torch

    mesh, parts = H.gpu_seed(wl, n_props=0)
    if kind is None:
        tape = P.pic_advect_record(parts.h, mesh.h, dt, integrator, steps)
    else:
        tape = P.pic_advect_record_tape(parts.h, mesh.h, dt, integrator, steps, kind)
    st = parts.export()
    ids = st["id"].cpu().numpy()
    x = st["x"].cpu().numpy()
    r = x - targets_by_id[:, ids]
    lam = 2.0 * r
    if weight_by_id is not None:
        lam = lam * weight_by_id[ids][None, :]
    dU = torch.empty((wl.dim, wl.U.shape[1]), dtype=torch.float64, device="cuda")
    P.pic_tape_adjoint(tape, torch.as_tensor(np.ascontiguousarray(lam), device="cuda"), dU, dx0)
    P.pic_destroy_tape(tape)
    loss = float((r * r).sum())
    return loss, dU.cpu().numpy(), ids, x, parts


def test_adjoint_matches_oracle_reverse_mode(P, oracle_mod):
    wl = W.curl_cube(6, 4, 4, 4, n_props=0)
    steps, dt = 4, 1.5 * wl.dt
    om, op = H.oracle_seed(oracle_mod, wl)
    tg = _targets_by_id(wl, op.n, op.x.T.copy())
    L_gpu, g_gpu, ids, x, _ = _gpu_grad(P, wl, steps, dt, 4, tg)
    L_orc, g_orc = oracle_mod.advect_adjoint(om, op, dt, 4, steps, tg.T[op.id.astype(np.int64)])
    assert L_gpu == pytest.approx(L_orc, rel=1e-12)
    scale = np.abs(g_orc).max()
    assert np.abs(g_gpu - g_orc).max() <= TOL_GRAD * scale, np.abs(g_gpu - g_orc).max() / scale


@pytest.mark.parametrize("integrator", [2, 1])
def test_adjoint_other_integrators_2d(P, oracle_mod, integrator):
    wl = W.c5_member(7, 12)
    steps, dt = 3, 2 * wl.dt
    om, op = H.oracle_seed(oracle_mod, wl)
    tg = _targets_by_id(wl, op.n, op.x.T.copy())
    L_gpu, g_gpu, ids, x, _ = _gpu_grad(P, wl, steps, dt, integrator, tg)
    L_orc, g_orc = oracle_mod.advect_adjoint(om, op, dt, integrator, steps, tg.T[op.id.astype(np.int64)])
    assert L_gpu == pytest.approx(L_orc, rel=1e-12)
    assert np.abs(g_gpu - g_orc).max() <= TOL_GRAD * np.abs(g_orc).max()


def test_adjoint_is_reproducible(P):
    wl = W.curl_cube(5, 6, 3, 8, n_props=0)
    tg = np.zeros((3, wl.n_particles)) + 0.5
    a = _gpu_grad(P, wl, 3, wl.dt, 4, tg)[1]
    b = _gpu_grad(P, wl, 3, wl.dt, 4, tg)[1]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["3d_rk4", "2d_rk2", "3d_losses"])
def test_checkpoint_tape_equals_stage_tape(P, case):
    """A checkpoint tape replays each step from the store at its start with
    the forward's own particle step, so dL/dU and dL/dx0 equal those of the
    stage tape bit for bit, also when particles leave through the walls."""
    import torch

    if case == "3d_rk4":
        wl, steps, dt, rk = W.curl_cube(6, 5, 4, 5, n_props=0), 4, None, 4
    elif case == "2d_rk2":
        wl, steps, dt, rk = W.c5_member(9, 31), 3, None, 2
    else:
        wl, steps, dt, rk = W.curl_cube(6, 6, 3, 9, n_props=0), 3, "12x", 4
    dt = 12 * wl.dt if dt == "12x" else wl.dt  # CFL ~6: about a sixth of the particles leave
    tg = _targets_by_id(wl, wl.n_particles, np.full((wl.dim, wl.n_particles), 0.5))
    out = {}
    for kind in (P.PIC_TAPE_STAGES, P.PIC_TAPE_CHECKPOINTS):
        dx0 = torch.empty((wl.dim, wl.n_particles), dtype=torch.float64, device="cuda")
        L, g, ids, x, parts = _gpu_grad(P, wl, steps, dt, rk, tg, kind=kind, dx0=dx0)
        out[kind] = (L, g, ids, x, dx0.cpu().numpy(), parts.state()[1])
    a, b = out[P.PIC_TAPE_STAGES], out[P.PIC_TAPE_CHECKPOINTS]
    assert a[0] == b[0]
    for k in (1, 2, 3, 4):
        np.testing.assert_array_equal(a[k], b[k])
    if case == "3d_losses":
        assert a[5] > 0  # some particles were lost
    assert np.abs(a[1]).max() > 0


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_when_every_particle_is_lost(P, kind):
    """All particles leave during the recorded run: no survivor, so dL/dU and
    dL/dx0 are zero, through either tape kind."""
    import torch

    wl = W.c1(n=4, ppc=2)
    mesh, parts = H.gpu_seed(wl, n_props=0)
    N0 = parts.state()[0]
    tape = P.pic_advect_record_tape(parts.h, mesh.h, 40.0, 4, 2, kind)
    assert parts.state()[0] == 0
    dU = torch.full((wl.dim, wl.U.shape[1]), 7.0, dtype=torch.float64, device="cuda")
    dx0 = torch.full((wl.dim, N0), 7.0, dtype=torch.float64, device="cuda")
    # dL/dx_final has no column; a one-column array stands in (the sweep reads no entry)
    P.pic_tape_adjoint(tape, torch.zeros((wl.dim, 1), dtype=torch.float64, device="cuda"), dU, dx0)
    P.pic_destroy_tape(tape)
    assert not dU.any() and not dx0.any()


def test_tape_kind_errors(P):
    wl = W.curl_cube(3, 2, 2, 2, n_props=0)
    mesh, parts = H.gpu_seed(wl, n_props=0)
    with pytest.raises(P.PicError):
        P.pic_advect_record_tape(parts.h, mesh.h, wl.dt, 4, 2, 7)
    with pytest.raises(P.PicError):
        P.pic_advect_record_tape(parts.h, mesh.h, wl.dt, 4, 0, P.PIC_TAPE_CHECKPOINTS)


def test_autograd_function(P):
    import torch

    wl = W.curl_cube(5, 4, 3, 6, n_props=0)
    tg = _targets_by_id(wl, wl.n_particles, np.full((3, wl.n_particles), 0.5))
    ref_loss, ref_g, _, _, _ = _gpu_grad(P, wl, 3, wl.dt, 4, tg)
    mesh, parts = H.gpu_seed(wl, n_props=0)
    U = torch.as_tensor(wl.U, device="cuda").clone().requires_grad_(True)
    x, ids = P.advect_differentiable(U, parts, wl.dt, P.PIC_RK4, 3)
    t = torch.as_tensor(tg, device="cuda")[:, ids]
    loss = ((x - t) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(ref_loss, rel=1e-14)
    assert np.array_equal(U.grad.cpu().numpy(), ref_g)
    # the same through a checkpoint tape
    mesh2, parts2 = H.gpu_seed(wl, n_props=0)
    U2 = torch.as_tensor(wl.U, device="cuda").clone().requires_grad_(True)
    x2, ids2 = P.advect_differentiable(U2, parts2, wl.dt, P.PIC_RK4, 3, tape_kind=P.PIC_TAPE_CHECKPOINTS)
    (((x2 - torch.as_tensor(tg, device="cuda")[:, ids2]) ** 2).sum()).backward()
    assert np.array_equal(U2.grad.cpu().numpy(), ref_g)


def test_c4_full_size(P, oracle_mod):
    """32^3 jittered hexes, 32 per cell (1,048,576 particles), RK4, 20 steps:
    (a) the gradient restricted to 200 sampled particles (dL/dx_final zero for
    the others) equals the oracle's reverse mode on those particles; (b) the
    full gradient matches central finite differences of the GPU forward loss
    on 16 random DOFs."""
    import torch

    wl = W.c4()
    steps, dt = wl.n_steps, wl.dt
    N = wl.n_particles
    # targets: the seeded initial positions (oracle seeding, in id order) plus
    # N(0, h^2) noise; the loss is then the squared displacement error
    om, op = H.oracle_seed(oracle_mod, wl)
    x0 = np.zeros((N, 3))
    x0[op.id.astype(np.int64)] = op.x
    tg = W.adjoint_targets(x0, 1.0 / 32, wl.seed).T.copy()
    # (a) sampled particles against the oracle
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(N, 200, replace=False))
    w = np.zeros(N)
    w[pick] = 1.0
    L, g_sample, ids, x, _ = _gpu_grad(P, wl, steps, dt, 4, tg, weight_by_id=w)
    sub = op.subset(pick)
    L_orc, g_orc = oracle_mod.advect_adjoint(om, sub, dt, 4, steps, tg.T[pick])
    assert np.abs(g_sample - g_orc).max() <= TOL_GRAD * np.abs(g_orc).max()
    # (b) finite differences of the GPU forward loss
    L0, g_full, _, _, _ = _gpu_grad(P, wl, steps, dt, 4, tg)

    def loss_at(U):
        m2 = P.Mesh(wl.n, wl.X, U)
        p2 = P.Particles(m2, uniform_count=wl.ppc, seed=wl.pseed)
        p2.advect(dt, 4, steps)
        e = p2.export()
        r = e["x"] - torch.as_tensor(tg, device="cuda")[:, e["id"]]
        v = float((r * r).sum())
        p2.close()
        m2.close()
        return v

    scale = np.abs(g_full).max()
    flat = rng.choice(g_full.size, 16, replace=False)
    h = 1e-4
    for q in flat:
        c, node = divmod(int(q), g_full.shape[1])
        Up = wl.U.copy()
        Up[c, node] += h
        Lp = loss_at(Up)
        Up[c, node] -= 2 * h
        Lm = loss_at(Up)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g_full[c, node]) <= 1e-5 * scale + 1e-4 * abs(g_full[c, node]), (q, fd, g_full[c, node])

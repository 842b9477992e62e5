"""Form 2 (batched ensemble): every problem of an ensemble matches its solo
run bit for bit (seeding, per-particle arithmetic and (cell, id) order are
the same code), in both run modes, through graph replay, across odd and even
step counts and after the autotuner; plus the oracle, and the bounded grid
barrier's failure path."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def _members(sides=(6, 9, 12, 5, 16), seed=40):
    return [W.c5_member(s, seed + q) for q, s in enumerate(sides)]


def _solo(P, wl, steps):
    mesh = P.Mesh(wl.n, wl.X, wl.U)
    parts = P.Particles(mesh, per_cell=wl.per_cell, seed=wl.pseed)
    if steps:
        parts.advect(wl.dt, 4, steps)
    e = parts.export()
    return {k: v.cpu().numpy() for k, v in e.items() if k != "props"}


def _ens(P, wls):
    meshes = [P.Mesh(w.n, w.X, w.U) for w in wls]
    ens = P.Ensemble(meshes, per_cell=[w.per_cell for w in wls], seeds=[w.pseed for w in wls])
    ens.set_dt([w.dt for w in wls])
    return ens, meshes


def _check_same(P, ens, wls, steps):
    for q, w in enumerate(wls):
        got = {k: v.cpu().numpy() for k, v in ens.export(q).items()}
        want = _solo(P, w, steps)
        np.testing.assert_array_equal(got["id"], want["id"])
        np.testing.assert_array_equal(got["cell"], want["cell"])
        np.testing.assert_array_equal(got["x"], want["x"])
        np.testing.assert_array_equal(got["xhat"], want["xhat"])


def test_barrier_wait_runs_out_and_context_survives(P):
    import torch

    assert P.pic_barrier_selftest(0.2) == P.PIC_ERR_TIMEOUT
    assert float(torch.ones(1000, device="cuda").sum()) == 1000.0


@pytest.mark.parametrize("mode,use_graph", [(0, False), (0, True), (1, False), (1, True)])
def test_ensemble_matches_solo_runs(P, mode, use_graph):
    wls = _members()
    ens, meshes = _ens(P, wls)
    _check_same(P, ens, wls, 0)
    ens.run(4, 3, mode=mode, use_graph=use_graph)  # odd: buffer parity flips
    _check_same(P, ens, wls, 3)
    ens.run(4, 2, mode=mode, use_graph=use_graph)
    ens.run(4, 2, mode=mode, use_graph=use_graph)  # replays a cached graph
    _check_same(P, ens, wls, 7)


def test_ensemble_against_oracle(P, oracle_mod):
    wls = _members(sides=(7, 11, 4), seed=70)
    ens, meshes = _ens(P, wls)
    ens.run(4, 4, mode=1)
    for q, w in enumerate(wls):
        got = {k: v.cpu().numpy() for k, v in ens.export(q).items()}
        om, op = H.oracle_seed(oracle_mod, w)
        op = oracle_mod.advect(om, op, w.dt, 4, 4)
        np.testing.assert_array_equal(got["id"], op.id)
        np.testing.assert_array_equal(got["cell"], op.cell)
        assert np.abs(got["x"].T - op.x).max() <= H.TOL_X


def test_autotuner_restores_state(P):
    wls = _members(sides=(20, 8, 30), seed=90)
    ens, meshes = _ens(P, wls)
    ens.run(4, 2, mode=0)
    before = [{k: v.cpu().numpy() for k, v in ens.export(q).items()} for q in range(len(wls))]
    b, t, ms = ens.tune(4)
    assert b >= 1 and t in (32, 128, 512) and ms > 0
    after = [{k: v.cpu().numpy() for k, v in ens.export(q).items()} for q in range(len(wls))]
    for a, c in zip(before, after):
        for k in a:
            np.testing.assert_array_equal(a[k], c[k])
    ens.run(4, 3, mode=1)
    _check_same(P, ens, wls, 5)
    ens.run(4, 2, mode=0)  # the per-step mode with the tuned tile
    _check_same(P, ens, wls, 7)


def test_c5_full_size(P):
    """The 64-member ensemble the benchmark runs (57M particles), 10 steps in
    one persistent launch: every member's count is conserved, and three
    members chosen across the size range equal their solo runs bit for bit."""
    wls = W.c5()
    ens, meshes = _ens(P, wls)
    ens.run(4, wls[0].n_steps, mode=1)
    sizes = [w.n[0] for w in wls]
    for q in sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), len(wls) // 2}):
        got = {k: v.cpu().numpy() for k, v in ens.export(q).items() if k != "props"}
        solo = _solo(P, wls[q], wls[q].n_steps)
        for k in ("id", "cell", "x", "xhat"):
            np.testing.assert_array_equal(got[k], solo[k])
    alive, lost = ens.state()[:2]
    assert alive + lost == sum(w.n_particles for w in wls)

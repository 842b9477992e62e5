"""The slab partition of one mesh (parallel transport, Sec. 2.4) on CPU: the
slab arithmetic, the sub-mesh slices, and the particle exchange protocol over
2 and 3 gloo ranks.  Each rank holds particles of its owned layers that have
moved (a random step of at most one layer), sorted by cell as after a time
step; the ranges below and above its layers go to the neighbours through
slab.swap_with_neighbours, and each rank keeps its own and adds what it
receives.  No GPU and no CUDA library are involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1612_03369_gb300 import slab
from paper_1612_03369_gb300 import workloads as W


def test_slab_bounds_cover_and_balance():
    for n2 in (4, 7, 64, 128):
        for world in range(1, min(n2, 9) + 1):
            b = slab.slab_bounds(n2, world)
            assert b[0][0] == 0 and b[-1][1] == n2
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab.slab_bounds(3, 4)


def test_sub_mesh_slices_and_numbering():
    n = (5, 4, 9)
    X = W.jittered_vertices(n, 3)
    U = np.arange(3 * 11 * 9 * 19, dtype=np.float64).reshape(3, -1)  # one value per (component, node)
    for world in (1, 2, 3):
        owned = np.zeros(n[2], dtype=int)
        for r in range(world):
            s = slab.make_slab(n, r, world, halo=2)
            owned[s.k_lo: s.k_hi] += 1
            assert s.g_lo == max(0, s.k_lo - 2) and s.g_hi == min(n[2], s.k_hi + 2)
            nz = s.g_hi - s.g_lo
            Xl = slab.slice_vertices(X, s)
            assert Xl.shape == (3, (n[0] + 1) * (n[1] + 1) * (nz + 1))
            # vertex (i, j, kl) of the slice is global vertex (i, j, g_lo + kl)
            Xg = X.reshape(3, n[2] + 1, n[1] + 1, n[0] + 1)
            np.testing.assert_array_equal(Xl.reshape(3, nz + 1, n[1] + 1, n[0] + 1), Xg[:, s.g_lo: s.g_hi + 1])
            Ul = slab.slice_nodes(U, s)
            Ug = U.reshape(3, 2 * n[2] + 1, 2 * n[1] + 1, 2 * n[0] + 1)
            np.testing.assert_array_equal(Ul.reshape(3, 2 * nz + 1, 2 * n[1] + 1, 2 * n[0] + 1),
                                          Ug[:, 2 * s.g_lo: 2 * s.g_hi + 1])
            # local cell = global cell - shift, owned cells [own_lo, own_hi)
            assert s.shift == n[0] * n[1] * s.g_lo
            assert s.own_hi - s.own_lo == s.owned_cells == n[0] * n[1] * (s.k_hi - s.k_lo)
            per = slab.owned_per_cell(s, 3)
            assert per.sum() == 3 * s.owned_cells and per[s.own_lo: s.own_hi].min() == 3
            assert slab.first_id(s, 3) == 3 * n[0] * n[1] * s.k_lo
        np.testing.assert_array_equal(owned, 1)  # every layer owned exactly once


def test_leaving_ranges():
    assert slab.leaving_ranges(0, 10, 10) == ((0, 0), (10, 0))
    assert slab.leaving_ranges(3, 8, 12) == ((0, 3), (8, 4))


N_PROPS = 2


def _rank_particles(s, per_layer, seed):
    """Particles of the owned layers after a step: each moved by at most one
    layer (so some now sit in the halo), returned sorted by local cell as a
    store is after a step."""
    import torch

    g = np.random.default_rng(seed)
    L = s.layer
    k = np.repeat(np.arange(s.k_lo, s.k_hi), per_layer)
    ids = (np.arange(len(k)) + 1000 * s.rank + 10**6).astype(np.int64)
    cell_g = k * L + g.integers(0, L, len(k))
    move = g.integers(-1, 2, len(k)) * (g.uniform(size=len(k)) < 0.3)
    cell_g = np.clip(cell_g + move * L, 0, s.n[2] * L - 1)  # walls keep particles inside
    local = cell_g - s.shift
    order = np.lexsort((ids, local))
    x = g.uniform(size=(3, len(k)))[:, order]
    d = {"x": torch.from_numpy(x), "xhat": torch.from_numpy(x * 0.5),
         "id": torch.from_numpy(ids[order]), "cell": torch.from_numpy(cell_g[order].astype(np.int32)),
         "props": torch.from_numpy(np.stack([ids[order] * 1.0, -ids[order] * 2.0])[:N_PROPS])}
    return d


def _slab_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        n = (4, 3, 12)
        s = slab.make_slab(n, rank, world, halo=2)
        mine = _rank_particles(s, per_layer=7, seed=rank)
        # host form of export_leaving: the store is sorted by cell, so the
        # particles below / above the owned layers are a prefix / suffix
        loc = mine["cell"].numpy().astype(np.int64) - s.shift
        off = np.concatenate([[0], np.cumsum(np.bincount(loc, minlength=s.layer * (s.g_hi - s.g_lo)))])
        (f0, c0), (f1, c1) = slab.leaving_ranges(int(off[s.own_lo]), int(off[s.own_hi]), len(loc))
        cut = lambda f, c: {k: v[..., f: f + c] for k, v in mine.items()}
        down, up = cut(f0, c0), cut(f1, c1)
        assert (loc[:c0] < s.own_lo).all() and (loc[f1:] >= s.own_hi).all()
        from_below, from_above = slab.swap_with_neighbours(down, up, rank, world, torch.device("cpu"))
        kept = cut(c0, f1 - c0)
        merged = slab.concat([kept, from_below, from_above])
        sent = {"down": down["id"].tolist(), "up": up["id"].tolist(), "all": mine["id"].tolist()}
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, s, {k: v.numpy() for k, v in merged.items()}, sent))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, repr(e), None, None))


def _free_port():
    so = socket.socket()
    so.bind(("127.0.0.1", 0))
    port = so.getsockname()[1]
    so.close()
    return port


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, s, merged, sent = q.get(timeout=180)
        assert not isinstance(s, str), s
        res[rank] = (s, merged, sent)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    all_ids = sorted(i for r in res for i in res[r][2]["all"])
    got_ids = []
    for r, (s, merged, sent) in res.items():
        L = s.layer
        k = merged["cell"].astype(np.int64) // L
        # after the exchange every rank holds only its own layers' particles
        assert ((k >= s.k_lo) & (k < s.k_hi)).all()
        # each payload travelled intact (the properties encode the id)
        np.testing.assert_array_equal(merged["props"][0], merged["id"] * 1.0)
        np.testing.assert_array_equal(merged["props"][1], -merged["id"] * 2.0)
        got_ids += merged["id"].tolist()
        # the ends of the chain send nothing outward
        if r == 0:
            assert sent["down"] == []
        if r == world - 1:
            assert sent["up"] == []
    # conservation: every particle is held by exactly one rank
    assert sorted(got_ids) == all_ids

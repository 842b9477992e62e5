"""The slab partition of one mesh (parallel transport, Sec. 2.4) on one GPU:
2 and 3 ranks emulated one after another in one process (each rank's step
runs alone; the exchange is a hand-over between the ranks' stores in place
of the messages).  Every rank holds a sub-mesh of its layers plus two halo
layers, advances its own particles, exports those that left its layers with
their cells (pic_export_range) and merges what its neighbours export
(pic_merge_particles).  The union of the ranks' stores must equal the
single-store run bit for bit: same ids, same cells, same positions and
reference coordinates, same properties."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import slab
from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _host(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _union(P, stores, slabs):
    rows = []
    for st, s in zip(stores, slabs):
        n = st.state()[0]
        e = _host(st.export_range(0, n, cell_shift=s.shift))
        rows.append(e)
    out = {k: np.concatenate([r[k] for r in rows], axis=-1) for k in rows[0]}
    order = np.lexsort((out["id"], out["cell"]))
    return {k: v[..., order] for k, v in out.items()}


@pytest.mark.parametrize("world", [2, 3])
def test_slab_partition_equals_single_store(world):
    import torch
    from paper_1612_03369_gb300 import pic as P

    wl = W.curl_cube(10, 8, 6, 2)
    # the single store
    mesh_g, ref = H.gpu_seed(wl)
    N = ref.state()[0]
    start = ref.export_range(0, N)
    ref.advect(wl.dt, P.PIC_RK4, wl.n_steps)
    r = _host(ref.export_range(0, ref.state()[0]))

    # the ranks: sub-meshes, and each rank's particles out of the same seeding
    slabs = [slab.make_slab(wl.n, k, world, halo=2) for k in range(world)]
    meshes, stores = [], []
    for s in slabs:
        m = P.Mesh(s.local_n, slab.slice_vertices(wl.X, s), slab.slice_nodes(wl.U, s))
        st = P.Particles(m, per_cell=np.zeros(s.layer * (s.g_hi - s.g_lo), dtype=np.uint32), seed=wl.pseed,
                         n_props=wl.n_props, capacity=N)
        layer = start["cell"].long() // s.layer
        mine = (layer >= s.k_lo) & (layer < s.k_hi)
        st.merge(s.own_lo, s.own_hi, {k: v[..., mine] for k, v in start.items()}, cell_shift=-s.shift)
        meshes.append(m)
        stores.append(st)
    assert sum(st.state()[0] for st in stores) == N
    moved = 0
    for step in range(wl.n_steps):
        out = []
        for st in stores:
            st.advect(wl.dt, P.PIC_RK4, 1)
        for st, s in zip(stores, slabs):
            out.append(slab.export_leaving(st, s))
        for k, (st, s) in enumerate(zip(stores, slabs)):
            from_below = out[k - 1][1] if k > 0 else None
            from_above = out[k + 1][0] if k + 1 < world else None
            moved += sum(0 if d is None else int(d["id"].shape[0]) for d in (from_below, from_above))
            slab.merge_incoming(st, s, from_below, from_above)
    assert moved > 0  # particles did cross the slabs' boundaries
    u = _union(P, stores, slabs)
    np.testing.assert_array_equal(u["id"], r["id"])
    np.testing.assert_array_equal(u["cell"], r["cell"])
    for k in ("x", "xhat", "props"):
        assert np.array_equal(u[k].view(np.uint64), r[k].view(np.uint64)), k
    for st, s in zip(stores, slabs):
        assert st.state()[2] == 0  # no status bit raised
        layer = (st.export_range(0, st.state()[0], cell_shift=s.shift)["cell"].long() // s.layer).cpu().numpy()
        assert ((layer >= s.k_lo) & (layer < s.k_hi)).all()

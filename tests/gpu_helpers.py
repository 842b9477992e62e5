"""Shared set-up for the GPU parity tests: run a workload through the C ABI
and through the CPU oracle on the same seeded inputs."""
import numpy as np

# Tolerances (FP64 form).  Positions: 1e-12 of the unit domain's extent;
# reference coordinates: 1e-12 relative to the cell size, i.e. the position
# tolerance divided by the smallest cell edge; cell averages: 1e-12.
TOL_X = 1e-12
TOL_AVG = 1e-12


def tol_xhat(wl):
    return TOL_X * max(wl.n) * 1.25


def gpu_seed(wl, n_props=None, capacity=0):
    from paper_1612_03369_gb300 import pic as P

    mesh = P.Mesh(wl.n, wl.X, wl.U)
    parts = P.Particles(mesh, per_cell=wl.per_cell, uniform_count=wl.ppc or 0, seed=wl.pseed,
                        first_id=wl.first_id, n_props=wl.n_props if n_props is None else n_props, capacity=capacity)
    st = parts.export()
    for q in range(min(parts.n_props, wl.dim)):
        parts.set_property(q, st["x"][q].contiguous())  # property q = initial coordinate q
    return mesh, parts


def gpu_state(parts):
    e = parts.export()
    return {
        "x": e["x"].cpu().numpy().T.copy(),
        "xhat": e["xhat"].cpu().numpy().T.copy(),
        "id": e["id"].cpu().numpy().astype(np.uint64),
        "cell": e["cell"].cpu().numpy().view(np.uint32).astype(np.int64),
        "props": e["props"].cpu().numpy().T.copy(),
    }


def oracle_seed(O, wl):
    om = O.Mesh(wl.n, wl.X, wl.U)
    op = O.seed_particles(om, per_cell=wl.per_cell, uniform_count=wl.ppc or 0, seed=wl.pseed, first_id=wl.first_id,
                          n_props=wl.n_props)
    for q in range(min(wl.n_props, wl.dim)):
        op.props[:, q] = op.x[:, q]
    return om, op


def assert_same_store(g, o, wl, tol_x=TOL_X):
    assert g["id"].shape[0] == o.n, (g["id"].shape[0], o.n)
    np.testing.assert_array_equal(g["id"], o.id)
    np.testing.assert_array_equal(g["cell"], o.cell)
    if o.n:
        dx = np.abs(g["x"] - o.x).max()
        assert dx <= tol_x, dx
        dxh = np.abs(g["xhat"] - o.xhat).max()
        assert dxh <= tol_xhat(wl), dxh
        if o.props.shape[1]:
            assert np.abs(g["props"][:, : o.props.shape[1]] - o.props).max() <= tol_x

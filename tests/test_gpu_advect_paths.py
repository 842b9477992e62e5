"""The advect kernel's two ways of reading the cells' blocks (staged in
shared memory by bulk copies, or through the read-only cache) and its two
paths for a particle (the fast path, or the full path for the particles that
need a rare one) run the same arithmetic: the stores they leave must agree
bit for bit, and agree with the oracle (Sec. 2.3, 2.4)."""
import numpy as np
import pytest

from gpu_helpers import gpu_seed, gpu_state, oracle_seed, assert_same_store

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_staged_and_cached_reads_agree_bit_for_bit(precision):
    from paper_1612_03369_gb300 import pic as P
    from paper_1612_03369_gb300 import workloads as W

    wl = W.curl_cube(16, 20, 6, 2)
    states = []
    for stage in (False, True):
        mesh, parts = gpu_seed(wl)
        P.pic_set_advect_staging(parts.h, stage)
        parts.advect(wl.dt, P.PIC_RK4, wl.n_steps, precision)
        states.append(gpu_state(parts))
        parts.close()
        mesh.close()
    a, b = states
    for k in ("id", "cell"):
        np.testing.assert_array_equal(a[k], b[k])
    for k in ("x", "xhat", "props"):
        assert np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)), k


def test_staged_reads_match_oracle(oracle_mod):
    from paper_1612_03369_gb300 import pic as P
    from paper_1612_03369_gb300 import workloads as W

    wl = W.curl_cube(8, 20, 6, 2)
    mesh, parts = gpu_seed(wl)
    P.pic_set_advect_staging(parts.h, True)
    parts.advect(wl.dt, P.PIC_RK4, wl.n_steps)
    g = gpu_state(parts)
    parts.close()
    mesh.close()
    om, op = oracle_seed(oracle_mod, wl)
    op = oracle_mod.advect(om, op, wl.dt, 4, wl.n_steps)
    assert_same_store(g, op, wl)


def test_all_cells_search_runs_and_matches_oracle(oracle_mod):
    """At 12x the CFL-0.5 step stage points jump several cells, past the
    vertex neighbours of their hint: the all-cells search runs (a6), and the
    cells, ids, order and positions are still the oracle's brute-force
    owners."""
    from paper_1612_03369_gb300 import pic as P
    from paper_1612_03369_gb300 import workloads as W

    wl = W.curl_cube(6, 12, 2, 5)
    dt = wl.dt * 12.0
    mesh, parts = gpu_seed(wl)
    s0 = parts.stats()
    parts.advect(dt, P.PIC_RK4, wl.n_steps)
    s1 = parts.stats()
    g = gpu_state(parts)
    parts.close()
    mesh.close()
    assert s1["global_searches"] > s0["global_searches"]
    assert s1["deferred"] > s0["deferred"]
    om, op = oracle_seed(oracle_mod, wl)
    op = oracle_mod.advect(om, op, dt, 4, wl.n_steps)
    assert_same_store(g, op, wl)

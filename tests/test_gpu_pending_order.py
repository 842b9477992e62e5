"""The rebin order that pic_advect leaves pending (applied inside the next
pic_advect, read through by the cell averages, applied first by every other
call): one-step calls give the same store as one multi-step call, bit for
bit; the averages read through the pending order equal the averages of the
settled store; and each kind of call that settles the order sees the sorted
store (export, set_properties, locate, transfers, export_range)."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _wl():
    return W.curl_cube(9, 8, 4, 31)


def _bits(parts):
    g = H.gpu_state(parts)
    return {k: (v.view(np.uint64) if v.dtype == np.float64 else v) for k, v in g.items()}


def _avgs(P, parts, n_props):
    out = []
    for q in range(n_props):
        for kind in (P.PIC_AVG_ARITHMETIC, P.PIC_AVG_HARMONIC):
            a, c = parts.average(q, kind=kind)
            out.append((a.cpu().numpy().view(np.uint64), c.cpu().numpy()))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_one_step_calls_equal_one_call(precision):
    wl = _wl()
    _, a = H.gpu_seed(wl)
    _, b = H.gpu_seed(wl)
    a.advect(wl.dt, 4, wl.n_steps, precision)
    for _ in range(wl.n_steps):
        b.advect(wl.dt, 4, 1, precision)
        b.average(0)  # reads through the pending order, leaves it pending
    sa, sb = _bits(a), _bits(b)
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)


def test_averages_through_pending_order_equal_settled():
    from paper_1612_03369_gb300 import pic as P

    wl = _wl()
    _, parts = H.gpu_seed(wl)
    parts.advect(wl.dt, 4, 2)
    pending = _avgs(P, parts, wl.n_props)
    parts.export()  # settles the order
    settled = _avgs(P, parts, wl.n_props)
    for (a1, c1), (a2, c2) in zip(pending, settled):
        np.testing.assert_array_equal(a1, a2)
        np.testing.assert_array_equal(c1, c2)


def test_calls_that_settle_see_the_sorted_store():
    import torch
    from paper_1612_03369_gb300 import pic as P

    wl = _wl()
    _, ref = H.gpu_seed(wl)
    ref.advect(wl.dt, 4, 2)
    want = _bits(ref)  # export settled it
    want_vavg = ref.vertex_average(0)[0].cpu().numpy()

    # set_properties writes slot order: property 1 := id of the slot
    _, p = H.gpu_seed(wl)
    p.advect(wl.dt, 4, 2)
    N = p.state()[0]
    ids = torch.from_numpy(want["id"].astype(np.float64)).cuda()
    p.set_property(1, ids)
    g = _bits(p)
    np.testing.assert_array_equal(g["id"], want["id"])
    np.testing.assert_array_equal(g["props"][:, 1].view(np.float64), want["id"].astype(np.float64))

    # the transfers and the range export read the sorted store
    _, p = H.gpu_seed(wl)
    p.advect(wl.dt, 4, 2)
    np.testing.assert_array_equal(p.vertex_average(0)[0].cpu().numpy(), want_vavg)
    _, p = H.gpu_seed(wl)
    p.advect(wl.dt, 4, 2)
    e = p.export_range(3, N - 5)
    np.testing.assert_array_equal(e["id"].cpu().numpy().astype(np.uint64), want["id"][3: N - 2])

    # locate re-sorts from the sorted store: nothing moves
    _, p = H.gpu_seed(wl)
    p.advect(wl.dt, 4, 2)
    p.locate()
    g = _bits(p)
    for k in ("id", "cell", "x"):
        np.testing.assert_array_equal(g[k], want[k], err_msg=k)

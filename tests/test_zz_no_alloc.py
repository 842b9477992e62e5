"""pic_sort_by_cell_noalloc, the sort entry point that allocates nothing.

It serves callers that cannot allocate device memory where they sort (their
own pool has reserved the device, their allocator must own every byte, or
they must not enter the driver's allocator).  Its scratch is a fixed array
inside the library, so these checks run it through the C ABI twice in a row,
with different inputs, and compare each result bit for bit with
pic_sort_by_cell (which allocates its scratch per call) on the same input;
the second call must not see anything left over from the first.  A call at
exactly both advertised limits must be accepted and match too; calls past a
limit must fail on the host and leave the outputs untouched.  The first test
makes the n = 0 call that loads the array on the device, as the header asks
of a caller.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOST = 0xFFFFFFFF


def _case(n, C, seed):
    g = np.random.default_rng(seed)
    cell = g.integers(0, C, n).astype(np.uint32)
    cell[g.uniform(size=n) < 0.05] = LOST
    ids = (g.permutation(4 * n)[:n].astype(np.uint64) * 3 + 1)
    return cell, ids


def _both(P, cell, ids, C):
    import torch

    tc = torch.as_tensor(cell.view(np.int32).copy(), device="cuda")
    ti = torch.as_tensor(ids.view(np.int64).copy(), device="cuda")
    ref_perm, ref_off = P.pic_sort_by_cell(tc, ti, C)
    perm = torch.full((max(len(cell), 1),), -7, dtype=torch.int32, device="cuda")
    off = torch.full((C + 1,), -7, dtype=torch.int32, device="cuda")
    P.pic_sort_by_cell_noalloc(tc, ti, C, perm, off)
    torch.cuda.synchronize()
    ref_off = ref_off.cpu().numpy()
    off = off.cpu().numpy()
    k = int(ref_off[-1])
    return ref_perm.cpu().numpy()[:k], ref_off, perm.cpu().numpy()[:k], off


def test_noalloc_warm_up_call_with_no_items():
    from paper_1612_03369_gb300 import pic as P
    import torch

    cell = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
    ids = torch.zeros(1, dtype=torch.int64, device="cuda")[:0]
    perm = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    off = torch.full((17,), -7, dtype=torch.int32, device="cuda")
    P.pic_sort_by_cell_noalloc(cell, ids, 16, perm, off)
    torch.cuda.synchronize()
    assert off.cpu().numpy().tolist() == [0] * 17
    assert int(perm.cpu()[0]) == -7


def test_noalloc_matches_allocating_sort_twice():
    from paper_1612_03369_gb300 import pic as P

    # first call: many items in few cells; second: fewer items in more cells,
    # so stale counts or keys from the first call would show
    for n, C, seed in ((400_000, 5_000, 1), (120_001, 90_000, 2)):
        cell, ids = _case(n, C, seed)
        ref_perm, ref_off, perm, off = _both(P, cell, ids, C)
        np.testing.assert_array_equal(off, ref_off)
        np.testing.assert_array_equal(perm, ref_perm)
        # and the order is the (cell, id) order
        keep = np.nonzero(cell < C)[0]
        np.testing.assert_array_equal(perm, keep[np.lexsort((ids[keep], cell[keep]))])


def test_noalloc_at_both_limits():
    from paper_1612_03369_gb300 import pic as P

    n, C = 524_288, 131_072  # the largest call the header accepts
    cell, ids = _case(n, C, 3)
    ref_perm, ref_off, perm, off = _both(P, cell, ids, C)
    np.testing.assert_array_equal(off, ref_off)
    np.testing.assert_array_equal(perm, ref_perm)
    keep = np.nonzero(cell < C)[0]
    np.testing.assert_array_equal(perm, keep[np.lexsort((ids[keep], cell[keep]))])


def test_noalloc_rejects_sizes_past_its_limits():
    from paper_1612_03369_gb300 import pic as P
    import torch

    big = torch.zeros(524_289, dtype=torch.int32, device="cuda")
    ids = torch.zeros(524_289, dtype=torch.int64, device="cuda")
    out = torch.full((524_289,), -7, dtype=torch.int32, device="cuda")
    off = torch.full((131_073 + 1,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PicError, match="limit"):
        P.pic_sort_by_cell_noalloc(big, ids, 10, out, off)
    small = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PicError, match="limit"):
        P.pic_sort_by_cell_noalloc(small, ids[:10], 131_073, out, off)
    torch.cuda.synchronize()
    # a refused call enqueues nothing: the outputs keep their fill
    assert bool((out == -7).all()) and bool((off == -7).all())

"""Stateless sort by (cell, id) through the C ABI against numpy's lexsort:
bit-exact permutation and offsets, including lost and out-of-range entries,
empty input, a single cell holding many items, and large ragged inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOST = 0xFFFFFFFF


def expected(cell, ids, C):
    keep = cell < C
    idx = np.nonzero(keep)[0]
    order = idx[np.lexsort((ids[idx], cell[idx]))]
    off = np.zeros(C + 1, dtype=np.int64)
    off[1:] = np.cumsum(np.bincount(cell[keep].astype(np.int64), minlength=C))
    return order, off


def make_case(n, C, seed, lost_frac=0.05, bad_frac=0.01, skew=False):
    g = np.random.default_rng(seed)
    if skew:
        cell = np.minimum(C - 1, (g.pareto(1.2, n) * 3).astype(np.int64)).astype(np.uint32)
    else:
        cell = g.integers(0, C, n).astype(np.uint32)
    r = g.uniform(size=n)
    cell[r < lost_frac] = LOST
    cell[(r >= lost_frac) & (r < lost_frac + bad_frac)] = C + 7
    ids = g.permutation(n * 3)[:n].astype(np.uint64) * 11 + 5
    return cell, ids


def run(P, cell, ids, C):
    import torch

    tc = torch.as_tensor(cell.view(np.int32).copy(), device="cuda")
    ti = torch.as_tensor(ids.view(np.int64).copy(), device="cuda")
    perm, off = P.pic_sort_by_cell(tc, ti, C)
    off = off.cpu().numpy().view(np.uint32).astype(np.int64)
    perm = perm.cpu().numpy().view(np.uint32).astype(np.int64)[: off[-1]]
    return perm, off


@pytest.mark.parametrize("n,C,skew", [(0, 5, False), (1, 1, False), (37, 1, False), (1000, 17, False),
                                      (300_001, 1000, False), (200_000, 50_000, True), (5000, 3, False)])
def test_sort_by_cell_matches_lexsort(n, C, skew):
    from paper_1612_03369_gb300 import pic as P

    cell, ids = make_case(n, C, seed=n + C, skew=skew)
    want_perm, want_off = expected(cell, ids, C)
    perm, off = run(P, cell, ids, C)
    np.testing.assert_array_equal(off, want_off)
    np.testing.assert_array_equal(perm, want_perm)


def test_sort_by_cell_argument_errors():
    from paper_1612_03369_gb300 import pic as P
    import torch

    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PicError):
        P.pic_sort_by_cell(t, torch.zeros(4, dtype=torch.int64, device="cuda"), 0)

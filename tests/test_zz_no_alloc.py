"""The allocation-free neighbour entry point (vct_build_neighbours_noalloc).

It exists for callers that cannot allocate device memory when they need
neighbour lists (their device memory belongs to their own pool, or cudaMalloc
is too costly in their loop).  The test calls it through the C ABI and checks
its CSR against the context-based vct_build_neighbours -- integer output, so
bit for bit -- over consecutive calls that reuse the shared static scratch.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def _reference(V, sc):
    solver = V.Solver(sc)
    row, col = solver.vct_build_neighbours(V.DeviceState(sc))
    out = row.cpu().numpy(), col.cpu().numpy()
    solver.close()
    return out


def _noalloc(V, sc, col_cap):
    import torch
    st = V.DeviceState(sc)
    row = torch.full((sc.n + 1,), -7, dtype=torch.int64, device="cuda")
    col = torch.full((max(col_cap, 1),), -7, dtype=torch.int32, device="cuda")
    rc, nnz = V.vct_build_neighbours_noalloc(sc, st, row, col)
    return rc, nnz, row.cpu().numpy(), col.cpu().numpy()[:nnz]


def test_noalloc_matches_context_entry_on_consecutive_calls():
    from paper_2607_28872_b300 import vct as V
    cases = [S.still_water_bf(),
             S.small_tank(dim=3, kind="SIGMA", L=0.15, W=0.11, H=0.07, d0=0.01, seed=5)]
    refs = [_reference(V, sc) for sc in cases]
    # two rounds over two scenarios of different dimension: every call reuses the
    # scratch the previous one left behind
    for _ in range(2):
        for sc, (rrow, rcol) in zip(cases, refs):
            rc, nnz, row, col = _noalloc(V, sc, rcol.size)
            assert rc == V.VCT_OK, V.vct_strerror(rc)
            assert nnz == rcol.size
            assert np.array_equal(row, rrow)
            assert np.array_equal(col, rcol)


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2607_28872_b300 import vct as V
    big = S.solitary_sigma()                       # 45,543 particles > 16,384
    rc, nnz, _, _ = _noalloc(V, big, 16)
    assert rc == V.VCT_ERR_CAPACITY
    sc = S.still_water_bf()
    rrow, rcol = _reference(V, sc)
    rc, nnz, _, _ = _noalloc(V, sc, rcol.size - 1)   # column capacity too small
    assert rc == V.VCT_ERR_CAPACITY and nnz == rcol.size


def test_noalloc_count_only_and_cell_limit():
    """col = NULL returns only nnz and row_ptr (the documented count-only
    form), equal to the context entry's; a box whose cell grid exceeds the
    32768-cell limit is rejected with VCT_ERR_CAPACITY before any launch."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.1, d0=0.01, seed=3)
    rrow, rcol = _reference(V, sc)
    st = V.DeviceState(sc)
    for _ in range(2):
        row = torch.full((sc.n + 1,), -7, dtype=torch.int64, device="cuda")
        rc, nnz = V.vct_build_neighbours_noalloc(sc, st, row, None)
        assert rc == V.VCT_OK, V.vct_strerror(rc)
        assert nnz == rcol.size
        assert np.array_equal(row.cpu().numpy(), rrow)
    # 0.024 m cells over a 20.1 m x 1.1 m box: 838 x 46 = 38,548 > 32,768 cells
    row = torch.zeros(sc.n + 1, dtype=torch.int64, device="cuda")
    rc, _ = V.vct_build_neighbours_noalloc(sc, st, row, None, box_lo=(-0.1, 0.0, -0.1),
                                           box_hi=(20.0, 0.0, 1.0))
    assert rc == V.VCT_ERR_CAPACITY

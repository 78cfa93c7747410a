"""The allocation-free binning entry point (md_bin_static).

Some callers may not allocate GPU memory (their framework owns it, or their
loop has a fixed budget); md_bin_static bins atoms using only a fixed array
inside the library.  This file is collected last so that, if it fails, a run
that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import chaingen
import paper_1001_3764_gb300 as md

pytestmark = pytest.mark.gpu


def test_static_binning_matches_the_system_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    md.load()
    melt = chaingen.melt(40, seed=31)
    s = md.System(melt, precision=md.MD_MIXED, rebin_every=4)
    s.step(5)
    s.rebin()
    x, _, _ = s.state()
    want_cell_of, want_start, want_perm = s.bins()
    M = s.info["cells_per_side"]
    n = len(x)
    pos = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()          # SoA [3][n]
    stream = torch.cuda.current_stream()
    for _ in range(2):                                                  # the scratch keeps the last call's contents
        cell_of = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        start = torch.full((M ** 3 + 1,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        md.md_bin_static(pos.data_ptr(), n, melt["L"], M, cell_of.data_ptr(), start.data_ptr(),
                         perm.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(cell_of.cpu().numpy(), want_cell_of)
        assert np.array_equal(start.cpu().numpy(), want_start)
        assert np.array_equal(perm.cpu().numpy(), want_perm)
    s.close()


@pytest.mark.parametrize("n,M,crowd", [(20000, 5, 0.7), (50000, 1, 1.0), (3000, 50, 0.0)])
def test_static_binning_crowded_cells(n, M, crowd):
    """Cells far above a melt's occupancy (14,000 atoms in one of 125 cells;
    50,000 atoms in a single cell) and a nearly empty grid: the order inside
    each cell is built in bounded work (sorted runs of 256, then merge
    passes) and must still be the stable order by atom index that the oracle's
    counting sort gives.  Two calls in a row, since the scratch keeps the
    last call's contents."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    md.load()
    L = 5.0
    rng = np.random.default_rng(n)
    x = rng.uniform(0.0, L, size=(n, 3))
    k = int(crowd * n)
    x[:k] = rng.uniform(0.0, 0.9 * L / M, size=(k, 3))     # inside cell 0
    want_cell_of, want_start, want_perm = oracle.bin_atoms(x, L, M)
    pos = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        cell_of = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        start = torch.full((M ** 3 + 1,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        md.md_bin_static(pos.data_ptr(), n, L, M, cell_of.data_ptr(), start.data_ptr(), perm.data_ptr(),
                         stream.cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(cell_of.cpu().numpy(), want_cell_of)
        assert np.array_equal(start.cpu().numpy(), want_start)
        assert np.array_equal(perm.cpu().numpy(), want_perm)


def test_static_binning_rejects_sizes_beyond_its_limits():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    md.load()
    with pytest.raises(md.MDError) as e:
        md.md_bin_static(1, (1 << 20) + 1, 10.0, 5, 1, 1, 1, 0)
    assert e.value.code == md.MD_EINVAL and "n_atoms" in md.md_last_error()
    with pytest.raises(md.MDError) as e:
        md.md_bin_static(1, 100, 10.0, 51, 1, 1, 1, 0)
    assert e.value.code == md.MD_EINVAL and "cells" in md.md_last_error()

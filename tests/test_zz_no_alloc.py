"""The allocation-free binning entry point gives the same result as the
scratch-buffer one.

crm_bin_points_noalloc exists for callers that cannot allocate device memory when
they bin (host callbacks, real-time loops, callers whose device memory belongs to
their own allocator): its scratch is a built-in device array shared by all calls.
This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

crm = pytest.importorskip("paper_2507_05643_b300")


def _points(seed, n, dims, cell, spread=1.0):
    rng = np.random.default_rng(seed)
    ext = np.array(dims, np.float32) * np.float32(cell)
    u = (rng.uniform(-0.02, 1.01, size=(n, 3)) - 0.5) * spread + 0.5
    return (u * ext).astype(np.float32)


def _bin_both(torch, xyz, dims, cell):
    dev = torch.device("cuda")
    n = xyz.shape[0]
    ncell = int(np.prod(dims))
    X = torch.from_numpy(xyz.reshape(-1)).to(dev) if n else torch.zeros(3, device=dev)
    outs = []
    for noalloc in (False, True):
        cells = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
        perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
        start = torch.full((ncell + 1,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        if noalloc:
            crm.bin_points_noalloc(X.data_ptr(), n, cell, dims, cells.data_ptr(), perm.data_ptr(),
                                   start.data_ptr())
        else:
            sb = crm.bin_scratch_bytes(n, ncell)
            scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
            crm.bin_points(X.data_ptr(), n, cell, dims, cells.data_ptr(), perm.data_ptr(),
                           start.data_ptr(), scratch.data_ptr(), sb)
        torch.cuda.synchronize()
        outs.append((cells.cpu().numpy(), perm.cpu().numpy(), start.cpu().numpy()))
    return outs


def _stable_reference(xyz, dims, cell):
    """The definition: clamped cell of each point, a stable argsort by cell and
    the start of each cell's run (NumPy on the host)."""
    cell = np.float32(cell)
    ijk = np.clip(np.floor(xyz * (np.float32(1.0) / cell)).astype(np.int64), 0,
                  np.array(dims) - 1)
    c = (ijk[:, 2] * dims[1] + ijk[:, 1]) * dims[0] + ijk[:, 0]
    perm = np.argsort(c, kind="stable")
    start = np.searchsorted(c[perm], np.arange(int(np.prod(dims)) + 1), side="left")
    return c, perm, start


def test_noalloc_matches_scratch_entry_point_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    cell = 0.024
    # different inputs back to back: each call must not see the previous one's
    # leftovers; an empty input; and one whose points lie ~90 % outside the grid,
    # clamped into a few boundary cells
    cases = ((1, 191_248, (88, 22, 29), 1.0), (2, 1_000_000, (160, 80, 60), 1.0),
             (3, 0, (5, 4, 3), 1.0), (4, 20_000, (16, 8, 8), 10.0))
    for seed, n, dims, spread in cases:
        xyz = _points(seed, n, dims, cell, spread)
        ref, got = _bin_both(torch, xyz, dims, cell)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)   # integer work: bit-exact
        c, perm, start = _stable_reference(xyz, dims, cell)
        assert np.array_equal(got[0][:n].astype(np.int64), c)
        assert np.array_equal(got[1][:n].astype(np.int64), perm)
        assert np.array_equal(got[2].astype(np.int64), start)


def test_noalloc_rejects_sizes_beyond_its_limits():
    with pytest.raises(crm.CrmError) as e:
        crm.bin_points_noalloc(256, (1 << 20) + 1, 0.1, (4, 4, 4), 256, 256, 256)
    assert e.value.code == -1
    with pytest.raises(crm.CrmError):
        crm.bin_points_noalloc(256, 10, 0.1, (1024, 1024, 1), 256, 256, 256)

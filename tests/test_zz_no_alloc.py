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


def _points(seed, n, dims, cell):
    rng = np.random.default_rng(seed)
    ext = np.array(dims, np.float32) * np.float32(cell)
    return (rng.uniform(-0.02, 1.01, size=(n, 3)) * ext).astype(np.float32)


def _bin_both(torch, xyz, dims, cell):
    dev = torch.device("cuda")
    n = xyz.shape[0]
    ncell = int(np.prod(dims))
    X = torch.from_numpy(xyz.reshape(-1)).to(dev)
    outs = []
    for noalloc in (False, True):
        cells = torch.full((n,), -1, dtype=torch.int32, device=dev)
        perm = torch.full((n,), -1, dtype=torch.int32, device=dev)
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


def test_noalloc_matches_scratch_entry_point_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    cell = 0.024
    # two different inputs back to back: the second call must not see the first's leftovers
    for seed, n, dims in ((1, 191_248, (88, 22, 29)), (2, 1_000_000, (160, 80, 60))):
        ref, got = _bin_both(torch, _points(seed, n, dims, cell), dims, cell)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)   # integer work: bit-exact


def test_noalloc_rejects_sizes_beyond_its_limits():
    with pytest.raises(crm.CrmError) as e:
        crm.bin_points_noalloc(256, (1 << 20) + 1, 0.1, (4, 4, 4), 256, 256, 256)
    assert e.value.code == -1
    with pytest.raises(crm.CrmError):
        crm.bin_points_noalloc(256, 10, 0.1, (1024, 1024, 1), 256, 256, 256)

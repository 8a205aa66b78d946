"""Failure detection of the bounded device waits (CRM_ETIMEOUT), exercised
without a GPU fault: crm_debug_wait_fault makes the look-back scans hold back
their first tile's prefix and give up each wait after a short bound, so the
waits of the later tiles run out and return with an error status that the host
reads.  Nothing hangs (every wait is bounded) and the context stays usable; the
next call after the switch is cleared is correct again."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

crm = pytest.importorskip("paper_2507_05643_b300")
import scenes  # noqa: E402


def test_stateless_binning_reports_a_wait_that_gave_up_and_recovers():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda")
    dims = (40, 30, 20)          # 24,000 cells: six tiles of the look-back scan
    ncell = int(np.prod(dims))
    cell = 0.024
    rng = np.random.default_rng(5)
    xyz = (rng.uniform(0, 1, size=(50_000, 3)) * np.array(dims) * cell).astype(np.float32)
    n = xyz.shape[0]
    X = torch.from_numpy(xyz.reshape(-1)).to(dev)
    cells = torch.zeros(n, dtype=torch.int32, device=dev)
    perm = torch.zeros(n, dtype=torch.int32, device=dev)
    start = torch.zeros(ncell + 1, dtype=torch.int32, device=dev)
    sb = crm.bin_scratch_bytes(n, ncell)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)

    def run(noalloc):
        start.fill_(0)
        torch.cuda.synchronize()
        if noalloc:
            crm.bin_points_noalloc(X.data_ptr(), n, cell, dims, cells.data_ptr(), perm.data_ptr(),
                                   start.data_ptr())
        else:
            crm.bin_points(X.data_ptr(), n, cell, dims, cells.data_ptr(), perm.data_ptr(),
                           start.data_ptr(), scratch.data_ptr(), sb)
        torch.cuda.synchronize()
        return start.cpu().numpy().view(np.uint32).copy(), perm.cpu().numpy().copy()

    good_start, good_perm = run(False)
    assert good_start[-1] == n
    for noalloc in (False, True):
        crm.debug_wait_fault(True)
        try:
            bad_start, _ = run(noalloc)
        finally:
            crm.debug_wait_fault(False)
        assert bad_start[-1] == 0xFFFFFFFF       # the timeout is reported
        s2, p2 = run(noalloc)                    # and the next call is right again
        assert np.array_equal(s2, good_start) and np.array_equal(p2, good_perm)


def test_terrain_reports_timeout_freezes_and_resumes_from_a_checkpoint():
    torch = pytest.importorskip("torch")
    # a bin large enough for a cell sort of several scan tiles
    sc = scenes.wheel_bin(seed=11, nx=60, ny=20, nz=8, wheel_radius=0.08, wheel_width=0.08,
                          n_grousers=6, wheel_x=0.2)
    # skin 0: every step sorts and searches, so the faulted steps run the scan
    ref = crm.from_scene(sc, skin=0.0)
    t = crm.from_scene(sc, skin=0.0)
    ref.step(sc.dt, 3)
    t.step(sc.dt, 3)
    t.sync()
    buf = torch.empty(t.state_bytes(), dtype=torch.uint8, device="cuda")
    used = t.save_state(buf.data_ptr(), buf.numel())
    x_before, _, _, _ = t.particles()
    crm.debug_wait_fault(True)
    try:
        t.step(sc.dt, 4)
        with pytest.raises(crm.CrmError) as e:
            t.sync()
    finally:
        crm.debug_wait_fault(False)
    assert e.value.code == -6      # CRM_ETIMEOUT
    # frozen: stepping is refused until a checkpoint is restored
    with pytest.raises(crm.CrmError) as e2:
        t.step(sc.dt, 1)
    assert e2.value.code == -8     # CRM_ESTATE
    d0 = sc.params["d0"]
    # resume from the checkpoint and follow the terrain that never failed
    t.load_state(buf.data_ptr(), used)
    t.step(sc.dt, 4)
    ref.step(sc.dt, 4)
    t.sync()
    xa, _, _, _ = t.particles()
    xb, _, _, _ = ref.particles()
    assert np.max(np.abs(xa - xb)) <= 1e-6 * d0
    assert np.max(np.abs(xb - x_before)) > 5e-6 * d0   # the run did move particles (1e-7 m)
    t.close()
    ref.close()

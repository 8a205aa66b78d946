"""The C-ABI library loads and exports every symbol include/crm.h declares, and its
host-side argument checks behave (no device work is issued by these calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "crm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2507_05643_b300 as crm
    names = _declared()
    assert len(names) >= 20
    lib = C.CDLL(crm.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(crm.EXPORTS)


def test_version_and_status_strings():
    import paper_2507_05643_b300 as crm
    assert crm.version() >= 100
    assert crm.lib().crm_status_string(-3) == b"CRM_ECAPACITY"


def test_default_params_match_paper_constants():
    import paper_2507_05643_b300 as crm
    p = crm.default_params()
    assert p.growth == pytest.approx(1.2) and p.shrink_ratio == pytest.approx(0.75)
    assert p.shrink_interval == 50
    assert p.ps_freq == 1 and p.av_mode == crm.AV_UNILATERAL


@pytest.mark.parametrize("field, value", [("rho0", 0.0), ("nu", 0.5), ("ps_freq", 0),
                                          ("max_neighbors", 4), ("h", -1.0), ("av_mode", 3),
                                          ("kernel", 2)])
def test_create_rejects_bad_params(field, value):
    import paper_2507_05643_b300 as crm
    p = crm.default_params()
    setattr(p, field, value)
    with pytest.raises(crm.CrmError) as e:
        crm.Terrain(p)
    assert e.value.code == -1


def test_add_rejects_out_of_domain_and_nonfinite():
    import paper_2507_05643_b300 as crm
    t = crm.Terrain(crm.default_params())
    with pytest.raises(crm.CrmError):
        t.add_sph(np.array([[0.5, 0.5, 1.5]]))
    with pytest.raises(crm.CrmError):
        t.add_sph(np.array([[0.5, np.nan, 0.5]]))
    with pytest.raises(crm.CrmError):
        t.add_rigid_body(np.zeros((1, 3)), [0.5, 0.5, 0.5, 1, 0, 0, 0], np.zeros(6), -1.0, 4)
    t.add_sph(np.array([[0.5, 0.5, 0.5]]))
    assert t.n_sph == 1
    with pytest.raises(crm.CrmError):
        t.step(-1.0, 1)
    t.close()


def test_bin_points_rejects_bad_arguments():
    import paper_2507_05643_b300 as crm
    with pytest.raises(crm.CrmError):
        crm.bin_points(0, 10, 0.1, (4, 4, 4), 0, 0, 0, 0, 0)
    with pytest.raises(crm.CrmError):
        crm.bin_points(256, 10, -0.1, (4, 4, 4), 256, 256, 256, 256, 1 << 20)
    assert crm.bin_scratch_bytes(1000, 64) >= 2 * 4 * 1000 + 4 * 65


def test_capacity_policy_matches_oracle():
    """ManageArrayMemory (Sec. 3.2): the library's capacity rule equals the oracle's
    on random need sequences, for the paper's G = 1.2, S = 0.75, S_I = 50 and others."""
    import numpy as np
    import oracle
    import paper_2507_05643_b300 as crm
    rng = np.random.default_rng(5)
    for G, S, SI in ((1.2, 0.75, 50), (1.5, 0.5, 7), (1.0, 1.0, 1)):
        cap_a = cap_b = 0
        for step in range(1, 400):
            need = int(rng.integers(0, 5000))
            cap_a = crm.capacity_policy(need, cap_a, step, G, S, SI)
            cap_b = oracle.capacity_policy(need, cap_b, step, G, S, SI)
            assert cap_a == cap_b
            assert cap_a >= need or step % SI == 0


def test_batch_rejects_members_without_their_own_stream():
    import paper_2507_05643_b300 as crm
    a = crm.Terrain(crm.default_params())
    b = crm.Terrain(crm.default_params())
    with pytest.raises(crm.CrmError):
        crm.Batch([a, b])              # both on the default stream
    with pytest.raises(crm.CrmError):
        crm.Batch([])
    with pytest.raises(crm.CrmError):
        a.set_pair_lanes(3)
    a.set_pair_lanes(1)
    a.close()
    b.close()


def test_adjoint_and_exchange_argument_checks():
    """The argument checks of the adjoint and co-simulation calls answer before any
    device work (no GPU needed)."""
    import paper_2507_05643_b300 as crm
    t = crm.Terrain(crm.default_params())
    t.add_sph(np.array([[0.5, 0.5, 0.5]]))
    with pytest.raises(crm.CrmError) as e:
        t.adjoint_backward()                       # nothing recorded
    assert e.value.code == -8                      # CRM_ESTATE
    for dt, n, every in ((-1.0, 2, 1), (1e-4, 0, 1), (1e-4, 2, -1)):
        with pytest.raises(crm.CrmError) as e:
            t.adjoint_forward(dt, n, every)
        assert e.value.code == -1                  # CRM_EINVAL
    lib = crm.lib()
    assert lib.crm_eval_rates_vjp(t._h, 0, None, None, None, 0, None, None, None, None, None,
                                  None, None) == -1   # capacity below the particle count
    assert lib.crm_cosim_step(t._h, np.zeros(7).ctypes.data, None, 1e-4, 1, None, None,
                              None) == -1          # a pose without a twist
    t.set_pair_lanes(4)
    t.set_pair_lanes(0)
    t.close()

"""The index-table check that runs on every plan before anything reaches the
device (no GPU needed: host-only plans run the same check).

Every plan the other tests build passes it; here the host fault-injection
hook (FMM_TEST_CORRUPT_TABLE) puts one out-of-range value into one table at
a time, and plan creation must refuse with FMM_ERR_UNSUPPORTED and name the
table, leaving nothing behind.
"""
import pytest

from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


TABLES = {"u_idx": "t.u_idx", "v_ptr": "v_ptr", "entry_src": "m.entry_src",
          "tile_target": "m.tile_target", "qidx": "t.qidx", "down_chunk": "down_chunk",
          "begin": "t.begin", "child": "t.child"}


@pytest.mark.parametrize("table", sorted(TABLES))
def test_planted_bad_index_is_refused(table, monkeypatch):
    x, _ = wl.gaussian_mixture(6000, 3)
    monkeypatch.setenv("FMM_TEST_CORRUPT_TABLE", table)
    with pytest.raises(N.FMMError) as e:
        FMMPlan(x, 4, 16, host_only=1)
    assert e.value.status == N.FMM_ERR_UNSUPPORTED
    assert "failed their check" in str(e.value) and TABLES[table] in str(e.value)
    monkeypatch.delenv("FMM_TEST_CORRUPT_TABLE")
    FMMPlan(x, 4, 16, host_only=1)          # the same input is sound


@pytest.mark.parametrize("kind,n,ncrit", [("cube", 1, 4), ("cube", 50, 64), ("sphere", 20000, 8),
                                          ("gauss", 30000, 12)])
def test_sound_plans_pass(kind, n, ncrit):
    gen = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture}
    x, _ = gen[kind](n, 4)
    FMMPlan(x, 4, ncrit, host_only=1)
    FMMPlan(x, 4, ncrit, host_only=1, balance=0)
    FMMPlan.batch([x, x[: max(1, n // 3)]], 4, ncrit, host_only=1)

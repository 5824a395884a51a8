"""The M2L work table of a plan against the plan's V lists (host-only plans).

The tensor-core and SIMT M2L kernels read nothing about the V lists but this
table, so every (target, source) V pair must appear in it exactly once, at
the offset index whose S_t translates from that source to that target
(S_t in lexicographic (tx, ty, tz) order over {-3..3}^3 minus {-1..1}^3), and
nothing else may.  The V lists themselves are checked against the oracle's
list definitions in test_abi_host.py and test_tree_levels.py.
"""
import numpy as np
import pytest

from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl

ROWS = 128
OFFSETS = np.array([(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)
                    if max(abs(a), abs(b), abs(c)) > 1], dtype=np.int64)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def check_table(P):
    keys = P.array("node_keys").reshape(-1, 4).astype(np.int64)
    prob = P.array("node_problem")
    vptr, vidx = P.array("v_ptr"), P.array("v_idx").astype(np.int64)
    lvl = P.array("m2l_tile_level")
    tgt = P.array("m2l_tile_target").reshape(-1, ROWS).astype(np.int64)
    eptr = P.array("m2l_tile_entry_ptr").astype(np.int64)
    eoff = P.array("m2l_entry_offset").astype(np.int64)
    esrc = P.array("m2l_entry_src").reshape(-1, ROWS).astype(np.int64)
    nt, ne = len(lvl), len(eoff)
    assert nt == P.info("m2l_tiles") and ne == P.info("m2l_entries")
    assert tgt.shape == (nt, ROWS) and len(eptr) == nt + 1 and esrc.shape == (ne, ROWS)
    assert eptr[0] == 0 and eptr[-1] == ne and np.all(np.diff(eptr) >= 1)

    # rows: filled from the first, one level and one parity class per tile
    filled = tgt >= 0
    cnt = filled.sum(1)
    assert np.all(cnt >= 1)
    assert np.array_equal(filled, np.arange(ROWS)[None, :] < cnt[:, None])
    assert np.all(lvl >= 2)
    tile_of_row = np.repeat(np.arange(nt), cnt)
    rows = tgt[filled]
    assert np.array_equal(keys[rows, 0], lvl[tile_of_row])
    cls = (keys[rows, 1] & 1) | ((keys[rows, 2] & 1) << 1) | ((keys[rows, 3] & 1) << 2)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    assert np.array_equal(cls, np.repeat(cls[first], cnt))

    # every box with a V list is the target of exactly one row, no other box
    vlen = np.diff(vptr)
    assert len(rows) == len(np.unique(rows))
    assert np.array_equal(np.sort(rows), np.flatnonzero(vlen > 0))
    # tiles follow (level, class) and, inside one, plan order
    order = np.lexsort((rows, cls, keys[rows, 0]))
    assert np.array_equal(order, np.arange(len(rows)))

    # entries: offsets increasing inside a tile, at most 189 per tile (one
    # parity class reaches 6^3 - 3^3 offsets), each used by some row
    tile_of_entry = np.repeat(np.arange(nt), np.diff(eptr))
    assert np.all((eoff >= 0) & (eoff < 316))
    same = tile_of_entry[1:] == tile_of_entry[:-1]
    assert np.all(eoff[1:][same] > eoff[:-1][same])
    assert np.diff(eptr).max() <= 189
    assert np.all((esrc >= 0).any(1))
    assert not np.any((esrc >= 0) & ~filled[tile_of_entry])

    # each (target, source, offset) of the table is a V pair at that offset
    e, r = np.nonzero(esrc >= 0)
    b, a = tgt[tile_of_entry[e], r], esrc[e, r]
    assert np.array_equal(keys[a, 0], keys[b, 0])
    assert np.array_equal(prob[a], prob[b])
    np.testing.assert_array_equal(keys[a, 1:] - keys[b, 1:], OFFSETS[eoff[e]])
    # ... and the table holds every V pair exactly once
    owner = np.repeat(np.arange(len(vlen)), vlen)
    nb = len(keys)
    want = np.sort(owner * nb + vidx)
    got = np.sort(b * nb + a)
    assert len(got) == P.info("v_pairs")
    np.testing.assert_array_equal(got, want)


CASES = [("cube", 10_000, 64, 1), ("cube", 60_000, 40, 1), ("sphere", 40_000, 32, 1),
         ("sphere", 40_000, 32, 0), ("gauss", 50_000, 24, 1), ("gauss", 50_000, 24, 0)]
GEN = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture}


@pytest.mark.parametrize("kind,n,ncrit,balance", CASES)
def test_m2l_table_holds_the_v_lists(kind, n, ncrit, balance):
    x, _ = GEN[kind](n, 7)
    P = FMMPlan(x, 4, ncrit, host_only=1, balance=balance)
    check_table(P)


def test_m2l_table_distinct_targets():
    x, _ = wl.gaussian_mixture(20_000, 8)
    y, _ = wl.uniform_cube(20_000, 9)
    check_table(FMMPlan(x, 4, 32, targets=y, host_only=1))


def test_m2l_table_of_a_forest():
    pts = [wl.uniform_cube(n, 20 + i)[0] for i, n in enumerate((3000, 40, 9000, 700))]
    check_table(FMMPlan.batch(pts, 4, 32, host_only=1))


def test_m2l_table_of_the_level_builder():
    x, _ = wl.sphere_surface(30_000, 10)
    check_table(FMMPlan(x, 4, 32, host_only=1, tree_build=N.TREE_LEVELS_HOST))


def test_m2l_table_empty_below_level_two():
    # one leaf: no box at level >= 2, so no tile
    x, _ = wl.uniform_cube(20, 11)
    P = FMMPlan(x, 4, 64, host_only=1)
    assert P.info("m2l_tiles") == 0 and P.info("m2l_entries") == 0
    assert len(P.array("m2l_tile_entry_ptr")) == 1


# ---------------------------------------------------------------------------
# the pair-column table (windows of target boxes, items of one offset)
# ---------------------------------------------------------------------------
WIN_TARGETS, ITEM_COLS = 256, 128


def check_windows(P, ncta=None):
    keys = P.array("node_keys").reshape(-1, 4).astype(np.int64)
    vptr, vidx = P.array("v_ptr"), P.array("v_idx").astype(np.int64)
    wtp, wt = P.array("m2l_win_target_ptr"), P.array("m2l_win_targets")
    wip, ioff = P.array("m2l_win_item_ptr"), P.array("m2l_item_offset")
    ipp, psrc, pslot = P.array("m2l_item_pair_ptr"), P.array("m2l_pair_src"), P.array("m2l_pair_slot")
    cptr, cwin = P.array("m2l_cta_ptr"), P.array("m2l_cta_win")
    nwin = len(wip) - 1
    assert nwin == P.info("m2l_windows") and len(ioff) == P.info("m2l_items")
    # windows cut the boxes with a V list, in plan order, into <= 256
    vlen = np.diff(vptr)
    assert np.array_equal(wt, np.flatnonzero(vlen > 0))
    assert wtp[0] == 0 and wtp[-1] == len(wt) and np.all(np.diff(wtp) >= 1)
    assert np.all(np.diff(wtp) <= WIN_TARGETS)
    # every window is dealt to exactly one block
    assert cptr[0] == 0 and cptr[-1] == nwin and np.all(np.diff(cptr) >= 0)
    assert np.array_equal(np.sort(cwin), np.arange(nwin))
    if ncta is not None:
        assert len(cptr) == ncta + 1
    # every V pair appears once, in its target's window, at the offset whose
    # S_t translates from the source to the target; items of a window in
    # increasing offset order, pairs in window order, at most 128 per item
    got = set()
    for w in range(nwin):
        tgt_of_slot = wt[wtp[w]:wtp[w + 1]]
        offs = ioff[wip[w]:wip[w + 1]]
        assert np.all(np.diff(offs) >= 0)
        for it in range(wip[w], wip[w + 1]):
            a, z = ipp[it], ipp[it + 1]
            assert 1 <= z - a <= ITEM_COLS
            sl = pslot[a:z]
            assert np.all(np.diff(sl) > 0) and sl.min() >= 0 and sl.max() < len(tgt_of_slot)
            tb = tgt_of_slot[sl]
            d = keys[psrc[a:z], 1:] - keys[tb, 1:]
            assert np.all(np.abs(d) <= 3) and np.all(np.abs(d).max(1) >= 2)
            np.testing.assert_array_equal(
                (d[:, 0] + 3) * 49 + (d[:, 1] + 3) * 7 + (d[:, 2] + 3),
                OFFSET_LEX[ioff[it]])
            for b, s in zip(tb, psrc[a:z]):
                assert (b, s) not in got
                got.add((b, s))
    want = {(b, s) for b in np.flatnonzero(vlen > 0) for s in vidx[vptr[b]:vptr[b + 1]]}
    assert got == want


OFFSET_LEX = np.array([(a + 3) * 49 + (b + 3) * 7 + (c + 3) for a, b, c in OFFSETS])


@pytest.mark.parametrize("gen,n,p,ncrit", [
    (wl.uniform_cube, 20_000, 4, 32),
    (wl.sphere_surface, 30_000, 4, 24),
    (wl.gaussian_mixture, 15_000, 4, 8),
], ids=["cube", "sphere", "gauss"])
def test_pair_column_windows_cover_every_v_pair(gen, n, p, ncrit):
    x, _ = gen(n, 11)
    P = FMMPlan(x, p, ncrit, host_only=1)
    check_windows(P, ncta=152)


def test_pair_column_windows_of_a_batch_and_of_a_plan_without_v_lists():
    xs = [wl.uniform_cube(m, 30 + m)[0] for m in (5000, 300, 12000)]
    check_windows(FMMPlan.batch(xs, 4, 32, host_only=1))
    P = FMMPlan(wl.uniform_cube(100, 3)[0], 4, 64, host_only=1)
    assert P.info("v_pairs") == 0 and P.info("m2l_windows") == 0
    check_windows(P)


def test_pair_column_windows_balance_the_blocks():
    x, _ = wl.sphere_surface(200_000, 12)
    P = FMMPlan(x, 4, 32, host_only=1)
    cptr = P.array("m2l_cta_ptr")
    per = np.diff(cptr)
    # a whole number of windows per block, so no block idles
    assert per.min() == per.max() >= 1
    check_windows(P, ncta=152)


def test_tile_schedule_deals_every_tile_once_and_balances():
    """The target-tile M2L's block schedule: with at least as many tiles as
    blocks, every tile goes to exactly one of the 152 blocks (host-only plans
    assume 152 SMs), longest first to the least loaded block, so the largest
    load exceeds the mean by less than the largest tile (cost: entries + 1);
    with fewer tiles there is no schedule (the kernel takes every gridDim-th
    tile)."""
    x, _ = wl.sphere_surface(200_000, 12)
    P = FMMPlan(x, 4, 32, host_only=1)
    eptr = P.array("m2l_tile_entry_ptr").astype(np.int64)
    cost = np.diff(eptr) + 1
    nt = len(cost)
    assert nt >= 152
    cptr = P.array("m2l_tile_cta_ptr").astype(np.int64)
    tiles = P.array("m2l_tile_cta_tiles").astype(np.int64)
    assert len(cptr) == 153 and cptr[0] == 0 and cptr[-1] == nt and np.all(np.diff(cptr) >= 1)
    assert np.array_equal(np.sort(tiles), np.arange(nt))
    load = np.array([cost[tiles[cptr[c]:cptr[c + 1]]].sum() for c in range(152)])
    assert load.max() - load.sum() / 152 < cost.max()
    # the round-robin order it replaces is worse on this adaptive tree
    rr = np.array([cost[c::152].sum() for c in range(152)])
    assert load.max() <= rr.max()
    small = FMMPlan(wl.uniform_cube(5000, 3)[0], 4, 64, host_only=1)
    assert small.info("m2l_tiles") < 152
    assert len(small.array("m2l_tile_cta_ptr")) == 0

"""Multi-rank partition of one problem (paper_2303_08394_gb300/partition.py),
on CPU with the gloo backend.

The partition cuts the Morton-ordered leaves into contiguous ranges of about
equal work, and lists what every rank must receive: upward densities of
boxes in its V and W lists that another rank completes, and the points of
U- and X-list leaves another rank owns (the locally essential tree).  The
test below runs the library's compressed scheme in FP64 (the same per-box
formulas as test_fp64_pipeline.run_fp64, from the plan's exported operators
and lists) on 2 and 3 gloo ranks: each rank starts with its own points only
(every other position and charge is NaN, so a missing piece of the
essential tree would show as NaN), computes the upward densities of the
boxes complete on it, all-gathers the frontier, forms the straddling top of
the tree, exchanges densities and points in one point-to-point round, and
evaluates its own points.  The potentials must equal the single-rank run.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")

from paper_2303_08394_gb300 import FMMPlan  # noqa: E402
from paper_2303_08394_gb300 import partition as pt  # noqa: E402
from paper_2303_08394_gb300 import workloads as wl  # noqa: E402

AI, AO = 1.05, 2.95
N, P_ORDER, NCRIT = 4000, 4, 24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def _problem():
    x, q = wl.gaussian_mixture(N, 5, nrhs=2)
    return x, q


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_and_balances():
    x, _ = _problem()
    P = FMMPlan(x, P_ORDER, NCRIT, host_only=1)
    tree = pt.Tree.from_plan(P)
    work = pt.leaf_work(tree, P.info("nsurf"))
    for world in (1, 2, 3, 5):
        part = pt.partition(tree, world, work, direct_max=P.info("nsurf"))
        leaves = np.flatnonzero(tree.leaf)
        assert np.all(part.owner[leaves] >= 0) and np.all(part.owner[~tree.leaf] == -1)
        # contiguous Morton ranges, ranks in order
        morton = leaves[np.argsort(tree.rng[leaves, 0])]
        assert np.all(np.diff(part.owner[morton]) >= 0)
        shares = np.array([work[part.owner == r].sum() for r in range(world)])
        assert shares.sum() == pytest.approx(work.sum())
        # each share within the largest single leaf of an equal split
        assert np.all(np.abs(shares - work.sum() / world) <= work.max() + 1e-9)
        # straddling boxes are exactly those whose leaves span ranks
        for b in range(len(tree.keys)):
            lo, hi = tree.rng[b]
            ranks = set(part.owner[[a for a in leaves if tree.rng[a, 0] >= lo
                                    and tree.rng[a, 1] <= hi]].tolist())
            assert (part.complete[b] >= 0) == (len(ranks) == 1)
        # sends mirror receives; nobody receives from itself
        for r in range(world):
            for s, ids in part.recv_up[r].items():
                assert s != r and np.array_equal(part.send_up(s)[r], ids)
                assert np.all(part.complete[ids] == s)
            for s, ids in part.recv_pts[r].items():
                assert s != r and np.array_equal(part.send_pts(s)[r], ids)
                assert np.all(part.owner[ids] == s)
        if world == 1:
            assert not part.recv_up[0] and not part.recv_pts[0]


def _k1(t, s):
    d = np.linalg.norm(t[:, None, :] - s[None, :, :], axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d > 0, 1.0 / d, 0.0)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from tests.test_fp64_pipeline import OFFSETS
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, q = _problem()
        P = FMMPlan(x, P_ORDER, NCRIT, host_only=1)
        tree = pt.Tree.from_plan(P)
        ns, rP, rQ, k = (P.info(a) for a in ("nsurf", "rank_up", "rank_down", "rank_m2l"))
        part = pt.partition(tree, world, pt.leaf_work(tree, ns), direct_max=ns)
        s = P.array("surface").reshape(ns, 3)
        Pu, Ps, Pv = (P.array("op_pu").reshape(ns, rP), P.array("op_ps"),
                      P.array("op_pv").reshape(ns, rP))
        Qu, Qs, Qv = (P.array("op_qu").reshape(ns, rQ), P.array("op_qs"),
                      P.array("op_qv").reshape(ns, rQ))
        M2M = P.array("op_m2m").reshape(8, rP, ns)
        L2L = P.array("op_l2l").reshape(8, rQ, ns)
        QUk = P.array("op_quk").reshape(rQ, k)
        Vk = P.array("m2l_v").reshape(ns, k)
        S = P.array("m2l_s").reshape(316, k, k)
        keys, rng, leaf = tree.keys, tree.rng, tree.leaf
        perm = P.array("perm")
        root = P.array("root")
        c0, hw = root[:3], root[3]
        h = hw / 2.0 ** keys[:, 0]
        cen = c0 - hw + (2 * keys[:, 1:] + 1) * h[:, None]
        sig = (keys[:, 1] & 1) | ((keys[:, 2] & 1) << 1) | ((keys[:, 3] & 1) << 2)
        index = {tuple(r_): i for i, r_ in enumerate(keys)}
        nrhs = q.shape[1]
        # this rank's points only; everything else unknown
        xs = np.full((len(x), 3), np.nan)
        qs = np.full((len(x), nrhs), np.nan)
        for b in np.flatnonzero(part.owner == rank):
            sl = slice(rng[b, 0], rng[b, 1])
            xs[sl], qs[sl] = x[perm[sl]], q[perm[sl]]

        def pts(b):
            return slice(rng[b, 0], rng[b, 1])

        def small(b):
            return leaf[b] and rng[b, 1] - rng[b, 0] <= ns

        def children(b):
            l = keys[b, 0]
            for sg in range(8):
                ch = index.get((l + 1, 2 * keys[b, 1] + (sg & 1), 2 * keys[b, 2] + (sg >> 1 & 1),
                                2 * keys[b, 3] + (sg >> 2 & 1)))
                if ch is not None:
                    yield sg, ch

        def upward(b, up):
            if leaf[b]:
                chk = Pu.T @ (_k1(AO * s, (xs[pts(b)] - cen[b]) / h[b]) @ qs[pts(b)])
            else:
                chk = np.zeros((rP, nrhs))
                for sg, ch in children(b):
                    chk += M2M[sg] @ up[ch]
            return Pv @ (chk / Ps[:, None])

        # 1. boxes complete on this rank, finest level first
        up = {}
        mine = np.flatnonzero(part.complete == rank)
        for b in mine[np.argsort(-keys[mine, 0], kind="stable")]:
            up[b] = upward(b, up)
        # 2. frontier densities to every rank, then the straddling top
        fr = [b for b in part.frontier if part.complete[b] == rank]
        packed = torch.from_numpy(np.concatenate([up[b].ravel() for b in fr])
                                  if fr else np.zeros(0))
        got = pt.allgather_variable(packed, rank, world)
        for r_ in range(world):
            ids = [b for b in part.frontier if part.complete[b] == r_]
            vals = got[r_].numpy().reshape(len(ids), ns, nrhs) if ids else []
            for b, v in zip(ids, vals):
                up[b] = v
        for b in part.straddling:
            up[b] = upward(b, up)
        # 3. one exchange: densities, then points and charges
        send = {d: torch.from_numpy(np.concatenate([up[b].ravel() for b in ids]))
                for d, ids in part.send_up(rank).items()}
        counts = {s_: len(ids) * ns * nrhs for s_, ids in part.recv_up[rank].items()}
        for s_, buf in pt.exchange(send, counts, rank, world, torch.float64).items():
            for b, v in zip(part.recv_up[rank][s_], buf.numpy().reshape(-1, ns, nrhs)):
                up[int(b)] = v
        width = 3 + nrhs
        send = {d: torch.from_numpy(np.concatenate(
                    [np.hstack([xs[pts(b)], qs[pts(b)]]).ravel() for b in ids]))
                for d, ids in part.send_pts(rank).items()}
        counts = {s_: sum(int(rng[b, 1] - rng[b, 0]) for b in ids) * width
                  for s_, ids in part.recv_pts[rank].items()}
        for s_, buf in pt.exchange(send, counts, rank, world, torch.float64).items():
            rows = buf.numpy().reshape(-1, width)
            o = 0
            for b in part.recv_pts[rank][s_]:
                c = int(rng[b, 1] - rng[b, 0])
                xs[pts(b)], qs[pts(b)] = rows[o:o + c, :3], rows[o:o + c, 3:]
                o += c
        # 4. downward pass over the local boxes, leaf pass over own leaves
        local = part.local(rank)
        V, W, U, X = tree.v, tree.w, tree.u, tree.x
        down = {}
        for l in range(2, keys[:, 0].max() + 1):
            for b in local[keys[local, 0] == l]:
                y = np.zeros((rQ, nrhs))
                if len(V[b]):
                    y += QUk @ sum(S[OFFSETS[tuple(keys[a, 1:] - keys[b, 1:])]] @ (Vk.T @ up[a])
                                   for a in V[b])
                if len(X[b]) and not small(b):
                    xchk = sum(_k1(AI * s, (xs[pts(a)] - cen[b]) / h[b]) @ qs[pts(a)]
                               for a in X[b])
                    y += Qu.T @ xchk
                if l >= 3:
                    par = index[(l - 1, keys[b, 1] // 2, keys[b, 2] // 2, keys[b, 3] // 2)]
                    y += L2L[sig[b]] @ down[par]
                down[b] = Qv @ (y / Qs[:, None])
        phi = {}
        for b in np.flatnonzero(part.owner == rank):
            xt = xs[pts(b)]
            acc = sum(_k1(xt, xs[pts(a)]) @ qs[pts(a)] for a in U[b]) / (4 * np.pi)
            if keys[b, 0] >= 2:
                acc = acc + _k1((xt - cen[b]) / h[b], AO * s) @ down[b] / (4 * np.pi * h[b])
            for a in W[b]:
                if small(a):
                    acc = acc + _k1(xt, xs[pts(a)]) @ qs[pts(a)] / (4 * np.pi)
                else:
                    acc = acc + _k1((xt - cen[a]) / h[a], AI * s) @ up[a] / (4 * np.pi * h[a])
            if small(b):
                for a in X[b]:
                    acc = acc + _k1(xt, xs[pts(a)]) @ qs[pts(a)] / (4 * np.pi)
            for i, row in zip(perm[pts(b)], acc):
                phi[int(i)] = row
        out[rank] = (phi, {s_: ids.tolist() for s_, ids in part.recv_up[rank].items()},
                     {s_: ids.tolist() for s_, ids in part.recv_pts[rank].items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_evaluation_equals_single_rank(world):
    import torch.multiprocessing as mp
    from tests.test_fp64_pipeline import run_fp64
    x, q = _problem()
    P = FMMPlan(x, P_ORDER, NCRIT, host_only=1)
    ref, _ = run_fp64(P, x, q)
    port = _free_port()
    with mp.Manager() as manager:
        out = manager.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    got = np.full_like(ref, np.nan)
    exchanged = 0
    for r in range(world):
        phi, rup, rpts = res[r]
        exchanged += sum(len(v) for v in rup.values()) + sum(len(v) for v in rpts.values())
        for i, row in phi.items():
            assert np.all(np.isnan(got[i]))  # every point evaluated by one rank
            got[i] = row
    assert exchanged > 0  # the ranks did depend on each other
    assert np.all(np.isfinite(got))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-13, err

"""Partition of one FMM problem over several ranks, and the data each rank
must receive (its locally essential tree), computed from a plan's exported
tree and interaction lists.

The scheme ("Parallelization strategies for FMM operators" generalised from
threads to ranks):

* The leaves, in Morton order (the order of their sorted point ranges), are
  cut into `world` contiguous ranges of about equal estimated work; a rank
  owns the points of its leaves.
* A box whose leaves all belong to one rank is *complete* on that rank,
  which computes its upward density.  The other boxes *straddle* ranks: the
  top of the tree.  Their children that are complete (the *frontier*) are
  sent to every rank (one all-gather), and every rank then forms the
  straddling boxes' densities itself, bottom up.
* A rank's *local* boxes are its leaves and all their ancestors.  It runs the
  downward pass over them and the leaf pass over its leaves.  For that it
  needs: the upward density of every box in V(b) (b local) and in W(b)
  (b a local leaf) that it does not already hold, and the points and charges
  of every leaf in U(b) (b a local leaf) and X(b) (b local) that another rank
  owns.  Both come from the owning rank in one variable-size exchange.  A
  W-list box that is a leaf of at most `direct_max` points acts through its
  points (the library's direct_wx rule), so its points are sent instead of
  its density.

This module holds only the host logic (no arithmetic of the method): the
partition, the per-rank receive and send lists, and the exchange itself over
``torch.distributed`` point-to-point calls (gloo on the host, NCCL between
device buffers).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _csr(ptr, idx):
    return [idx[ptr[b]:ptr[b + 1]] for b in range(len(ptr) - 1)]


@dataclass
class Tree:
    """The parts of a plan's exported arrays the partition reads."""
    keys: np.ndarray      # nodes x 4 (level, ix, iy, iz)
    rng: np.ndarray       # nodes x 2 sorted point range
    leaf: np.ndarray      # nodes, bool
    u: list
    v: list
    w: list
    x: list

    @classmethod
    def from_plan(cls, P):
        keys = P.array("node_keys").reshape(-1, 4).astype(np.int64)
        return cls(keys=keys, rng=P.array("node_range").reshape(-1, 2),
                   leaf=P.array("leaf_flag").astype(bool),
                   u=_csr(P.array("u_ptr"), P.array("u_idx")),
                   v=_csr(P.array("v_ptr"), P.array("v_idx")),
                   w=_csr(P.array("w_ptr"), P.array("w_idx")),
                   x=_csr(P.array("x_ptr"), P.array("x_idx")))

    def parents(self):
        """Parent node of every node (-1 for the root)."""
        index = {tuple(k): i for i, k in enumerate(self.keys)}
        par = np.full(len(self.keys), -1, dtype=np.int64)
        for i, (l, a, b, c) in enumerate(self.keys):
            if l > 0:
                par[i] = index[(l - 1, a // 2, b // 2, c // 2)]
        return par


def leaf_work(tree: Tree, nsurf: int) -> np.ndarray:
    """Estimated cost of each leaf's evaluation: the pairs of its leaf pass
    (near field over U, L2P and the W surfaces), as the leaf kernel counts
    them.  Zero for boxes that are not leaves."""
    npts = (tree.rng[:, 1] - tree.rng[:, 0]).astype(np.int64)
    work = np.zeros(len(npts), dtype=np.float64)
    for b in np.flatnonzero(tree.leaf):
        near = sum(int(npts[a]) for a in tree.u[b])
        surf = (int(tree.keys[b, 0] >= 2) + len(tree.w[b])) * nsurf
        work[b] = float(npts[b]) * (near + surf)
    return work


@dataclass
class Partition:
    world: int
    owner: np.ndarray         # nodes: rank owning the leaf, -1 for other boxes
    complete: np.ndarray      # nodes: rank holding all the box's leaves, -1 if it straddles
    parent: np.ndarray
    frontier: np.ndarray      # complete boxes whose parent straddles
    straddling: np.ndarray    # boxes whose leaves lie on several ranks, finest level first
    recv_up: list = field(default_factory=list)    # per rank: {source rank: box ids}
    recv_pts: list = field(default_factory=list)   # per rank: {source rank: leaf ids}

    def local(self, rank):
        """Boxes on the paths of the rank's leaves (leaves and ancestors)."""
        out = set()
        for b in np.flatnonzero(self.owner == rank):
            while b >= 0 and b not in out:
                out.add(int(b))
                b = int(self.parent[b])
        return np.array(sorted(out), dtype=np.int64)

    def send_up(self, rank):
        """{destination rank: box ids} the rank sends upward densities for."""
        return {r: d[rank] for r, d in enumerate(self.recv_up) if rank in d}

    def send_pts(self, rank):
        """{destination rank: leaf ids} whose points and charges it sends."""
        return {r: d[rank] for r, d in enumerate(self.recv_pts) if rank in d}


def partition(tree: Tree, world: int, work: np.ndarray | None = None,
              direct_max: int = -1) -> Partition:
    """Cut the Morton-ordered leaves into `world` ranges of about equal work
    and list what each rank receives.  Deterministic: every rank computes the
    same partition from the same plan.  direct_max: W-list leaves of at most
    this many points are needed as points (the plan's surface size when its
    direct_wx option is on, else -1)."""
    nn = len(tree.keys)
    leaves = np.flatnonzero(tree.leaf)
    leaves = leaves[np.argsort(tree.rng[leaves, 0], kind="stable")]  # Morton order
    wl = (work[leaves] if work is not None
          else (tree.rng[leaves, 1] - tree.rng[leaves, 0]).astype(np.float64))
    wl = np.maximum(wl, 1e-9)
    cum = np.cumsum(wl)
    # leaf i goes to the rank whose share of the total work holds its midpoint
    mid = (cum - 0.5 * wl) / cum[-1]
    rank_of = np.minimum((mid * world).astype(np.int64), world - 1)
    owner = np.full(nn, -1, dtype=np.int64)
    owner[leaves] = rank_of

    parent = tree.parents()
    # complete: the single rank of all leaves below, or -1; bottom up
    lo = np.full(nn, world, dtype=np.int64)
    hi = np.full(nn, -1, dtype=np.int64)
    lo[leaves] = rank_of
    hi[leaves] = rank_of
    for b in np.argsort(-tree.keys[:, 0], kind="stable"):
        p = parent[b]
        if p >= 0:
            lo[p] = min(lo[p], lo[b])
            hi[p] = max(hi[p], hi[b])
    complete = np.where(lo == hi, lo, -1)
    strad = np.flatnonzero(complete < 0)
    strad = strad[np.argsort(-tree.keys[strad, 0], kind="stable")]
    frontier = np.array([b for b in range(nn) if complete[b] >= 0 and parent[b] >= 0
                         and complete[parent[b]] < 0], dtype=np.int64)

    part = Partition(world=world, owner=owner, complete=complete, parent=parent,
                     frontier=frontier, straddling=strad)
    known_everywhere = set(strad.tolist()) | set(frontier.tolist())
    for r in range(world):
        loc = part.local(r)
        mine = set(np.flatnonzero(owner == r).tolist())
        need_up, need_pts = set(), set()
        for b in loc:
            need_up.update(int(a) for a in tree.v[b])
            need_pts.update(int(a) for a in tree.x[b])
            if tree.leaf[b]:
                for a in tree.w[b]:
                    a = int(a)
                    if tree.leaf[a] and tree.rng[a, 1] - tree.rng[a, 0] <= direct_max:
                        need_pts.add(a)
                    else:
                        need_up.add(a)
                need_pts.update(int(a) for a in tree.u[b])
        up_from, pts_from = {}, {}
        for a in sorted(need_up):
            s = int(complete[a])
            if s == r or a in known_everywhere:
                continue
            up_from.setdefault(s, []).append(a)
        for a in sorted(need_pts - mine):
            pts_from.setdefault(int(owner[a]), []).append(a)
        part.recv_up.append({s: np.array(v, dtype=np.int64) for s, v in up_from.items()})
        part.recv_pts.append({s: np.array(v, dtype=np.int64) for s, v in pts_from.items()})
    return part


def exchange(send: dict, recv_counts: dict, rank: int, world: int, dtype, device="cpu"):
    """One variable-size exchange: `send` maps a destination rank to a 1-D
    tensor, `recv_counts` maps a source rank to the element count expected
    from it.  Returns {source rank: tensor}.  Point-to-point sends and
    receives (gloo has no all-to-all); on NCCL the same calls move device
    buffers, which land in this rank's own memory."""
    import torch
    import torch.distributed as dist
    reqs, out = [], {}
    for s, n in sorted(recv_counts.items()):
        if s == rank or n == 0:
            continue
        buf = torch.empty(int(n), dtype=dtype, device=device)
        out[s] = buf
        reqs.append(dist.irecv(buf, src=s))
    for d, t in sorted(send.items()):
        if d == rank or t.numel() == 0:
            continue
        reqs.append(dist.isend(t.contiguous(), dst=d))
    for q in reqs:
        q.wait()
    return out


def allgather_variable(t, rank: int, world: int):
    """All-gather of one 1-D tensor per rank, the lengths differing: the
    lengths first, then the tensors padded to the longest.  Returns the list
    of every rank's tensor, this rank's included."""
    import torch
    import torch.distributed as dist
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    pad = torch.zeros(m, dtype=t.dtype, device=t.device)
    pad[:t.numel()] = t
    bufs = [torch.empty(m, dtype=t.dtype, device=t.device) for _ in range(world)]
    dist.all_gather(bufs, pad)
    return [b[:s] for b, s in zip(bufs, sizes)]

"""FP64 CPU kernel-independent FMM (KIFMM) for the Laplace kernel, dense M2L.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing in the CUDA
library imports, links or calls this module, and it uses nothing from the
library.

What it computes, in the paper's order ("The Fast Multipole Method" and
"Computational structure of FMM operators" sections):

* the octree: the root cube is split into 8 equal children, recursively,
  while a box holds more than ``ncrit`` points; optionally 2:1 balanced
  ("balance condition", same section);
* the interaction lists U, V, W, X that feed the near field, M2L, M2P and
  P2L;
* check and equivalent surfaces with n_e = n_c = 6(p-1)^2 + 2 points;
* P2M and M2M (bottom-up), then M2L over V, P2L over X and L2L (top-down
  from level 2), then near field over U, L2P and M2P at the leaves.  Every
  operator is a kernel evaluation followed by a pseudo-inverse of a
  check-to-equivalent matrix, exactly as written, with no compression.
* With ``direct_wx`` (the default, as in the library) a leaf with no more
  points than a surface interacts through its points in the W and X lists:
  as a W-list box of leaf B its points act on B's points directly (no
  M2P), and as a box with an X list it takes the X leaves' points directly
  (no P2L).  The sum is the same; those terms become exact.

Readings where the paper is silent (each is also listed in the design
notes of the repository):

* Root: smallest axis-aligned cube around all points, centred on the bounding
  box centre, half-width inflated by a relative 1e-6.  All points coincide:
  half-width 0.5.
* Point-to-box map: integer coordinate floor((x - corner) / (2 hw) * 2^16),
  clamped to [0, 2^16 - 1]; a box at level l holds the points whose
  coordinate shifted right by 16 - l equals its index.  A point on a split
  plane goes to the upper child.
* Splitting creates all 8 children; empty children stay in the tree during
  construction and balancing (so the balance condition is the usual one over
  all leaves), and boxes with no points below them are then dropped from
  every list and every operator (their expansions are zero).
* Lists, for boxes A, B that hold points ("adjacent" = closed boxes touch):
  U(B), B a leaf: leaves adjacent to B, B included.
  V(B), level >= 2: children of the boxes adjacent to B's parent at the
        parent's level (the parent included) that are not adjacent to B.
  W(B), B a leaf: descendants A of B's same-level adjacent boxes such that A
        is not adjacent to B but A's parent is.
  X(B): all A with B in W(A).
* Surfaces: the grid points of {-1, -1 + 2/(p-1), ..., 1}^3 on the boundary
  of [-1,1]^3 in lexicographic (a, b, c) order, c fastest.  Box (c, h):
  c + alpha h s.  Upward equivalent and downward check surfaces use
  alpha_inner = 1.05, upward check and downward equivalent surfaces
  alpha_outer = 2.95.
* Pseudo-inverses: numpy SVD-based pinv, singular values below
  rcond * sigma_max dropped.  Default rcond = 1e-7: in FP64 it leaves the
  error at p <= 7 unchanged against smaller cutoffs, while the cutoff 1e-14
  loses accuracy from p = 8 on (the explicit inverse then carries
  eps * 4e12 of rounding).
* Self-interaction (i != j in Eq. (1)): a pair at distance exactly zero is
  skipped.

Parity pins (tests/test_oracle_kifmm.py, tests/test_oracle_tree.py):
N <= ncrit reduces to the direct sum; every (target leaf, source leaf) pair
is accounted for exactly once by the lists; list-size bounds on balanced
trees; linearity in the charges; invariance under dyadic translation; 1/s
scaling; error against the direct sum falls with p; each operator's output
reproduces the field it represents.  The absolute error level at a given p
is parity unpinned: the paper prints no error figure.
"""
from __future__ import annotations

import itertools

import numpy as np

FOUR_PI = 4.0 * np.pi
KEY_BITS = 16          # integer coordinates at level 16 (finest level)


# ----------------------------------------------------------------------------
# kernel and surfaces
# ----------------------------------------------------------------------------

def laplace_kernel(targets, sources):
    """Matrix G[i, j] = 1 / (4 pi |t_i - s_j|), zero where t_i == s_j (Eq. 1)."""
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    s = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    d = t[:, None, :] - s[None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    out = np.zeros_like(r)
    nz = r > 0.0
    out[nz] = 1.0 / (FOUR_PI * r[nz])
    return out


def laplace_gradient_kernel(targets, sources):
    """Eq. (1) differentiated in the target (the paper evaluates potentials only;
    a reading for the gradient extension).  G[i, j, :] = (s_j - t_i) / (4 pi |t_i - s_j|^3): the gradient of
    laplace_kernel's entry with respect to the target position t_i; zero
    where t_i == s_j."""
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    s = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    d = s[None, :, :] - t[:, None, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    w = np.zeros_like(r)
    nz = r > 0.0
    w[nz] = 1.0 / (FOUR_PI * r[nz] ** 3)
    return d * w[:, :, None]


def surface_grid(p: int):
    """Unit-cube surface points: grid {-1, -1+2/(p-1), ..., 1}^3 on the
    boundary of [-1, 1]^3, lexicographic in (a, b, c) with c fastest.
    Count 6(p-1)^2 + 2 ("Computational structure of FMM operators")."""
    if p < 2:
        raise ValueError("p must be >= 2")
    pts = []
    for a in range(p):
        for b in range(p):
            for c in range(p):
                if min(a, b, c) == 0 or max(a, b, c) == p - 1:
                    pts.append([-1.0 + 2.0 * a / (p - 1),
                                -1.0 + 2.0 * b / (p - 1),
                                -1.0 + 2.0 * c / (p - 1)])
    return np.array(pts, dtype=np.float64)


def pinv(matrix, rcond=1e-7):
    """Check-to-equivalent inversion ("Computational structure of FMM
    operators": expansions from check potentials; the method is silent on
    the cutoff, a reading).  Pseudo-inverse through the SVD, dropping sigma < rcond * sigma_max."""
    return np.linalg.pinv(matrix, rcond=rcond)


# ----------------------------------------------------------------------------
# octree
# ----------------------------------------------------------------------------

def _adjacent(ka, kb):
    """Adjacency, on which every interaction list rests ("Computational
    structure of FMM operators").  Closed boxes ka, kb (level, i, j, k) touch or overlap."""
    la, lb = ka[0], kb[0]
    L = max(la, lb)
    sa, sb = L - la, L - lb
    for d in range(1, 4):
        lo_a, hi_a = ka[d] << sa, (ka[d] + 1) << sa
        lo_b, hi_b = kb[d] << sb, (kb[d] + 1) << sb
        if lo_a > hi_b or lo_b > hi_a:
            return False
    return True


def _parent(key):
    """The box one level up ("The Fast Multipole Method": each box is one of
    its parent's 8 equal parts)."""
    l, i, j, k = key
    return (l - 1, i >> 1, j >> 1, k >> 1)


def _children(key):
    """The 8 equal parts of a box ("The Fast Multipole Method")."""
    l, i, j, k = key
    return [(l + 1, 2 * i + cx, 2 * j + cy, 2 * k + cz)
            for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]


class Octree:
    """Linear octree over a point set ("Data-oriented design" section):
    boxes are keys (level, i, j, k); ``points[key]`` holds the indices of the
    points inside the box (for internal boxes too)."""

    def __init__(self, points, ncrit: int, max_level: int = KEY_BITS,
                 balance: bool = True):
        x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
        if len(x) == 0:
            raise ValueError("empty point set")
        if max_level > KEY_BITS:
            raise ValueError("max_level too large")
        self.x = x
        self.ncrit = int(ncrit)
        self.max_level = int(max_level)
        lo, hi = x.min(axis=0), x.max(axis=0)
        self.centre = 0.5 * (lo + hi)
        hw = 0.5 * float(np.max(hi - lo)) * (1.0 + 1e-6)
        self.half_width = hw if hw > 0.0 else 0.5
        self.corner = self.centre - self.half_width
        u = (x - self.corner) / (2.0 * self.half_width)
        icoord = np.floor(u * float(1 << KEY_BITS)).astype(np.int64)
        self.icoord = np.clip(icoord, 0, (1 << KEY_BITS) - 1)

        self.points = {}
        self.leaf = {}
        stack = [((0, 0, 0, 0), np.arange(len(x)))]
        while stack:
            key, idx = stack.pop()
            self.points[key] = idx
            if len(idx) > self.ncrit and key[0] < self.max_level:
                self._split(key, stack)
            else:
                self.leaf[key] = True
        if balance:
            self._balance()
        self.nonempty = {k for k, v in self.points.items() if len(v) > 0}
        self.leaves = sorted(k for k in self.nonempty if self.leaf[k])
        self.depth = max(k[0] for k in self.nonempty)

    def _split(self, key, stack=None):
        """("The Fast Multipole Method": a box is subdivided into 8 equal parts
        while it holds more than ncrit points.)  Create all 8 children of ``key`` and hand them its points."""
        l = key[0]
        idx = self.points[key]
        self.leaf[key] = False
        bits = (self.icoord[idx] >> (KEY_BITS - l - 1)) & 1
        for child in _children(key):
            cx, cy, cz = child[1] & 1, child[2] & 1, child[3] & 1
            sel = idx[(bits[:, 0] == cx) & (bits[:, 1] == cy) & (bits[:, 2] == cz)]
            if stack is None:
                self.points[child] = sel
                self.leaf[child] = True
            else:
                stack.append((child, sel))

    def _balance(self):
        """The balance condition of "Computational structure of FMM
        operators" (neighbouring leaves at most twice as large as each other).
        Refine leaves until adjacent leaves differ by at most one level.
        A leaf at level l violates the condition exactly when an internal box
        at level l+1 touches it."""
        changed = True
        while changed:
            changed = False
            for key in [k for k, v in self.leaf.items() if v]:
                l, i, j, k = key
                if l >= self.max_level:
                    continue
                must_split = False
                for a in range(2 * i - 1, 2 * i + 3):
                    for b in range(2 * j - 1, 2 * j + 3):
                        for c in range(2 * k - 1, 2 * k + 3):
                            if (2 * i <= a <= 2 * i + 1 and 2 * j <= b <= 2 * j + 1
                                    and 2 * k <= c <= 2 * k + 1):
                                continue
                            nb = (l + 1, a, b, c)
                            if nb in self.leaf and not self.leaf[nb]:
                                must_split = True
                                break
                        if must_split:
                            break
                    if must_split:
                        break
                if must_split:
                    self._split(key)
                    changed = True

    # geometry -----------------------------------------------------------
    def box_half_width(self, level):
        """Half-width of the boxes of a level: the root's halved once per level
        ("The Fast Multipole Method")."""
        return self.half_width / float(1 << level)

    def box_centre(self, key):
        """Centre of a box from its level and integer coordinates."""
        l = key[0]
        h = self.box_half_width(l)
        return self.corner + (2.0 * np.array(key[1:], dtype=np.float64) + 1.0) * h

    def is_leaf(self, key):
        """Whether the box was left unsplit by the splitting and the balancing."""
        return self.leaf[key]


# ----------------------------------------------------------------------------
# interaction lists
# ----------------------------------------------------------------------------

def _colleagues(tree, key):
    """Non-empty boxes at the same level touching ``key`` (``key``
    included): the same-level neighbours the lists of "Computational
    structure of FMM operators" are built from."""
    l, i, j, k = key
    out = []
    for a, b, c in itertools.product((-1, 0, 1), repeat=3):
        nb = (l, i + a, j + b, k + c)
        if nb in tree.nonempty:
            out.append(nb)
    return out


def build_lists(tree):
    """The U, V, W and X lists of "Computational structure of FMM
    operators" (the inputs of the near field, M2L, M2P and P2L).  U, V, W, X lists (dicts: box -> sorted list of boxes), as defined in
    the module docstring."""
    leaves = tree.leaves
    U, V, W, X = {}, {}, {}, {}
    # U: brute force over all leaves
    la = np.array(leaves, dtype=np.int64)
    if len(la):
        lev = la[:, 0]
        for b in leaves:
            L = np.maximum(lev, b[0])
            sa = L - lev
            sb = L - b[0]
            ok = np.ones(len(la), dtype=bool)
            for d in range(1, 4):
                lo_a, hi_a = la[:, d] << sa, (la[:, d] + 1) << sa
                lo_b, hi_b = b[d] << sb, (b[d] + 1) << sb
                ok &= (lo_a <= hi_b) & (lo_b <= hi_a)
            U[b] = sorted(tuple(int(v) for v in row) for row in la[ok])
    # V
    for b in tree.nonempty:
        if b[0] < 2:
            continue
        out = []
        for col in _colleagues(tree, _parent(b)):
            if tree.leaf[col]:
                continue
            for ch in _children(col):
                if ch in tree.nonempty and not _adjacent(ch, b):
                    out.append(ch)
        if out:
            V[b] = sorted(out)
    # W (and X as its inverse)
    for b in leaves:
        out = []
        for col in _colleagues(tree, b):
            if col == b or tree.leaf[col]:
                continue
            stack = [ch for ch in _children(col) if ch in tree.nonempty]
            while stack:
                d = stack.pop()
                if not _adjacent(d, b):
                    out.append(d)          # parent is adjacent by construction
                elif not tree.leaf[d]:
                    stack.extend(ch for ch in _children(d) if ch in tree.nonempty)
        if out:
            W[b] = sorted(out)
            for a in out:
                X.setdefault(a, []).append(b)
    for a in X:
        X[a].sort()
    return U, V, W, X


# ----------------------------------------------------------------------------
# the FMM
# ----------------------------------------------------------------------------

class KIFMM:
    """Dense FP64 KIFMM on an :class:`Octree`.

    ``evaluate(charges)`` returns potentials in the caller's point order and
    keeps every operator's output in attributes for per-operator tests:
    ``up`` (upward equivalent densities), ``down`` (downward equivalent
    densities), ``down_check`` (downward check potentials), ``m2l_check``
    (the V-list part of each downward check potential, the M2L's output),
    ``near`` and ``far`` (potentials split by source).
    """

    def __init__(self, points, p: int, ncrit: int, alpha_inner=1.05,
                 alpha_outer=2.95, rcond=1e-7, balance=True,
                 max_level=KEY_BITS, direct_wx=True):
        self.tree = Octree(points, ncrit, max_level=max_level, balance=balance)
        # small W / X leaves interact through their points (see evaluate)
        self.direct_wx = bool(direct_wx)
        self.p = int(p)
        self.alpha_inner = float(alpha_inner)
        self.alpha_outer = float(alpha_outer)
        self.rcond = float(rcond)
        self.surf = surface_grid(self.p)
        self.U, self.V, self.W, self.X = build_lists(self.tree)
        # check-to-equivalent pseudo-inverses, one pair per level
        self.uc2e, self.dc2e = {}, {}
        for l in range(2, self.tree.depth + 1):
            h = self.tree.box_half_width(l)
            k_up = laplace_kernel(self.alpha_outer * h * self.surf,
                                  self.alpha_inner * h * self.surf)
            k_dn = laplace_kernel(self.alpha_inner * h * self.surf,
                                  self.alpha_outer * h * self.surf)
            self.uc2e[l] = pinv(k_up, self.rcond)
            self.dc2e[l] = pinv(k_dn, self.rcond)
        self._m2l_cache = {}

    # surfaces of a box ----------------------------------------------------
    def _surface(self, key, alpha):
        """Check or equivalent surface of a box ("Computational structure of
        FMM operators": 6(p-1)^2 + 2 points): the unit surface scaled by
        alpha times the half-width and moved to the box centre."""
        h = self.tree.box_half_width(key[0])
        return self.tree.box_centre(key) + alpha * h * self.surf

    def _m2l_matrix(self, b, a):
        """The M2L's kernel evaluation between surfaces ("Computational
        structure of FMM operators": M2L over V).  K(DC_b, UE_a).  It depends only on the level and the integer offset
        a - b, so it is computed once per (level, offset) from that offset
        (a memo, not a change of the arithmetic)."""
        l = b[0]
        off = (a[1] - b[1], a[2] - b[2], a[3] - b[3])
        key = (l,) + off
        m = self._m2l_cache.get(key)
        if m is None:
            h = self.tree.box_half_width(l)
            shift = 2.0 * h * np.array(off, dtype=np.float64)
            m = laplace_kernel(self.alpha_inner * h * self.surf,
                               shift + self.alpha_inner * h * self.surf)
            self._m2l_cache[key] = m
        return m

    def evaluate(self, charges, gradient=False):
        """The operators in the order of "The Fast Multipole Method" (bottom-up,
        then top-down) and "Computational structure of FMM operators" (M2L and
        L2L from level 2 down, then near field, L2P and M2P at the leaves).
        Potentials at the points; with gradient=True also their gradients
        with respect to the target position, (n, 3) or (n, nrhs, 3): the
        leaf step applies the target-gradient of the kernel to the same
        sources and densities (near field over U, L2P, M2P); the upward and
        downward passes do not change."""
        t = self.tree
        q = np.asarray(charges, dtype=np.float64)
        vec = q.ndim == 1
        q = q.reshape(len(t.x), -1)
        nrhs = q.shape[1]
        ne = len(self.surf)
        ai, ao = self.alpha_inner, self.alpha_outer

        def small(key):
            """A leaf with no more points than a surface: as a W-list box it
            acts on the leaf through its points (instead of M2P), and as the
            target of an X list it takes the X leaves' points directly
            (instead of P2L); either way the same sum, evaluated exactly."""
            return self.direct_wx and t.is_leaf(key) and len(t.points[key]) <= ne

        # P2M: leaf sources -> upward check potential -> upward density
        up = {}
        for b in t.leaves:
            if b[0] < 2:
                continue
            idx = t.points[b]
            check = laplace_kernel(self._surface(b, ao), t.x[idx]) @ q[idx]
            up[b] = self.uc2e[b[0]] @ check
        # M2M: children densities -> parent check potential -> parent density
        for l in range(t.depth - 1, 1, -1):
            for b in sorted(k for k in t.nonempty if k[0] == l and not t.leaf[k]):
                check = np.zeros((ne, nrhs))
                uc = self._surface(b, ao)
                for ch in _children(b):
                    if ch in t.nonempty:
                        check += laplace_kernel(uc, self._surface(ch, ai)) @ up[ch]
                up[b] = self.uc2e[l] @ check
        # downward pass from level 2: M2L (V), P2L (X), L2L (parent)
        down, down_check, m2l_check = {}, {}, {}
        for l in range(2, t.depth + 1):
            for b in sorted(k for k in t.nonempty if k[0] == l):
                check = np.zeros((ne, nrhs))
                for a in self.V.get(b, ()):
                    check += self._m2l_matrix(b, a) @ up[a]
                if b in self.V:
                    m2l_check[b] = check.copy()
                if b in self.X and not small(b):
                    dc = self._surface(b, ai)
                    for a in self.X[b]:
                        idx = t.points[a]
                        check += laplace_kernel(dc, t.x[idx]) @ q[idx]
                par = _parent(b)
                if par[0] >= 2:
                    check += laplace_kernel(self._surface(b, ai),
                                            self._surface(par, ao)) @ down[par]
                down_check[b] = check
                down[b] = self.dc2e[l] @ check
        # leaves: near field (U), L2P (own local density), M2P (W)
        near = np.zeros((len(t.x), nrhs))
        far = np.zeros((len(t.x), nrhs))
        grad = np.zeros((len(t.x), nrhs, 3)) if gradient else None

        def apply(tidx, xt, srcs, dens, acc):
            acc[tidx] += laplace_kernel(xt, srcs) @ dens
            if gradient:
                grad[tidx] += np.einsum("ijk,jr->irk", laplace_gradient_kernel(xt, srcs), dens)

        for b in t.leaves:
            tidx = t.points[b]
            xt = t.x[tidx]
            for a in self.U[b]:
                sidx = t.points[a]
                apply(tidx, xt, t.x[sidx], q[sidx], near)
            if b[0] >= 2:
                apply(tidx, xt, self._surface(b, ao), down[b], far)
            for a in self.W.get(b, ()):
                if small(a):
                    sidx = t.points[a]
                    apply(tidx, xt, t.x[sidx], q[sidx], far)
                else:
                    apply(tidx, xt, self._surface(a, ai), up[a], far)
            if small(b):
                for a in self.X.get(b, ()):
                    sidx = t.points[a]
                    apply(tidx, xt, t.x[sidx], q[sidx], far)
        self.up, self.down, self.down_check = up, down, down_check
        self.m2l_check = m2l_check
        self.near, self.far = near, far
        phi = near + far
        phi = phi[:, 0] if vec else phi
        if not gradient:
            return phi
        return phi, (grad[:, 0, :] if vec else grad)


def fmm(points, charges, p, ncrit, **kw):
    """One-call FP64 KIFMM: potentials of Eq. (1) at the points."""
    return KIFMM(points, p, ncrit, **kw).evaluate(charges)

"""A host-only FP64 run of the library's compressed scheme against the dense
FP64 oracle (no GPU needed).

The run below takes the library's own precomputed operators (exported by
fmm_plan_get_array: the factored check-to-equivalent pseudo-inverses, the
composite M2M and L2L, U_k, V_k, S_t, Q_u^T U_k) and the plan's tree and
lists, and walks the library's data flow in FP64 numpy: P2M and M2M through
Pv diag(1/Ps) Pu^T, the projection V_k^T, the compressed M2L S_t, the
downward pass through Qv diag(1/Qs) (Q_u^T U_k chat + Q_u^T P2L + L2L), and
the leaf step (near field, L2P, M2P).  Everything is in the unit-box form
the kernels use: in box B's coordinates y' = (y - c_B) / h_B a density rho
generates sum_j rho_j / |y' - a s_j| / (4 pi h_B).

With eps_svd = 0 (dense M2L) this must reproduce the oracle to FP64
rounding; with the compressed M2L to within a small multiple of eps_svd.
A wrong composite (a missing 1/2 in L2L, a transposed factor, a wrong
child centre or offset order) shows as an O(1) error.
"""
import itertools

import numpy as np
import pytest

from oracle import kifmm as ok
from paper_2303_08394_gb300 import FMMPlan
from paper_2303_08394_gb300 import workloads as wl

AI, AO = 1.05, 2.95
OFFSETS = {t: i for i, t in enumerate(
    t for t in itertools.product(range(-3, 4), repeat=3) if max(map(abs, t)) > 1)}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def k1(t, s):
    """1/|t_i - s_j|, 0 where they coincide."""
    d = np.linalg.norm(t[:, None, :] - s[None, :, :], axis=2)
    with np.errstate(divide="ignore"):
        return np.where(d > 0, 1.0 / d, 0.0)


def csr(P, name):
    ptr, idx = P.array(name + "_ptr"), P.array(name + "_idx")
    return [idx[ptr[b]:ptr[b + 1]] for b in range(len(ptr) - 1)]


def run_fp64(P, x, q, plant=None):
    """Potentials (n, nrhs) and the per-box intermediates of the library's
    scheme, in FP64, from the plan's exported operators and lists.  plant
    puts one known mistake into this run (for the sensitivity test):
    "l2l_child" takes the L2L block of the child mirrored in x, "s_transpose"
    applies S_t transposed."""
    ns, rP, rQ, k = (P.info(a) for a in ("nsurf", "rank_up", "rank_down", "rank_m2l"))
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
    if plant == "s_transpose":
        S = S.transpose(0, 2, 1)
    keys = P.array("node_keys").reshape(-1, 4).astype(np.int64)
    rng = P.array("node_range").reshape(-1, 2)
    leaf = P.array("leaf_flag").astype(bool)
    perm = P.array("perm")
    root = P.array("root")
    c0, hw = root[:3], root[3]
    U, V, W, X = (csr(P, a) for a in "uvwx")
    nn = len(keys)
    h = hw / 2.0 ** keys[:, 0]
    cen = c0 - hw + (2 * keys[:, 1:] + 1) * h[:, None]
    sig = (keys[:, 1] & 1) | ((keys[:, 2] & 1) << 1) | ((keys[:, 3] & 1) << 2)
    index = {tuple(r): i for i, r in enumerate(keys)}
    xs, qs = x[perm], q[perm]
    nrhs = q.shape[1]

    def pts(b):
        return slice(rng[b, 0], rng[b, 1])

    def small(b):
        # a leaf with no more points than a surface takes part in W and X
        # lists through its points (the plan's default direct_wx rule)
        return leaf[b] and rng[b, 1] - rng[b, 0] <= ns

    up, qhat, chat, down = {}, {}, {}, {}
    k_p2m = lambda b: k1(AO * s, (xs[pts(b)] - cen[b]) / h[b]) @ qs[pts(b)]
    for l in range(keys[:, 0].max(), 1, -1):
        for b in np.flatnonzero(keys[:, 0] == l):
            if leaf[b]:
                chk = Pu.T @ k_p2m(b)
            else:
                chk = np.zeros((rP, nrhs))
                for sg in range(8):
                    ch = index.get((l + 1, 2 * keys[b, 1] + (sg & 1), 2 * keys[b, 2] + (sg >> 1 & 1),
                                    2 * keys[b, 3] + (sg >> 2 & 1)))
                    if ch is not None:
                        chk += M2M[sg] @ up[ch]
            up[b] = Pv @ (chk / Ps[:, None])
            qhat[b] = Vk.T @ up[b]
    for b in range(nn):
        if len(V[b]):
            chat[b] = sum(S[OFFSETS[tuple(keys[a, 1:] - keys[b, 1:])]] @ qhat[a] for a in V[b])
    for l in range(2, keys[:, 0].max() + 1):
        for b in np.flatnonzero(keys[:, 0] == l):
            y = np.zeros((rQ, nrhs))
            if b in chat:
                y += QUk @ chat[b]
            if len(X[b]) and not small(b):
                xchk = sum(k1(AI * s, (xs[pts(a)] - cen[b]) / h[b]) @ qs[pts(a)] for a in X[b])
                y += Qu.T @ xchk
            if l >= 3:
                par = index[(l - 1, keys[b, 1] // 2, keys[b, 2] // 2, keys[b, 3] // 2)]
                y += L2L[sig[b] ^ (plant == "l2l_child")] @ down[par]
            down[b] = Qv @ (y / Qs[:, None])
    phi = np.zeros((len(x), nrhs))
    for b in np.flatnonzero(leaf):
        xt = xs[pts(b)]
        acc = sum(k1(xt, xs[pts(a)]) @ qs[pts(a)] for a in U[b]) / (4 * np.pi)
        if keys[b, 0] >= 2:
            acc = acc + k1((xt - cen[b]) / h[b], AO * s) @ down[b] / (4 * np.pi * h[b])
        for a in W[b]:
            if small(a):
                acc = acc + k1(xt, xs[pts(a)]) @ qs[pts(a)] / (4 * np.pi)
            else:
                acc = acc + k1((xt - cen[a]) / h[a], AI * s) @ up[a] / (4 * np.pi * h[a])
        if small(b):
            for a in X[b]:
                acc = acc + k1(xt, xs[pts(a)]) @ qs[pts(a)] / (4 * np.pi)
        phi[perm[pts(b)]] = acc
    return phi, dict(up=up, chat=chat, down=down, keys=keys, h=h, s=s,
                     Uk=P.array("m2l_u").reshape(ns, k))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (name, generator, n, p, ncrit, nrhs, eps_svd, bar).  eps_svd = 0 keeps
# K_t dense (FP64 rounding only: 4e-13 and 2.4e-11 measured); at p = 6
# eps_svd = 5e-7 keeps k = 127 of 152 singular values and 1e-6 keeps 116,
# and the truncation costs about 2-2.5 eps_svd in the M2L's check potentials
# (9.1e-7 and 2.5e-6 measured): the bar is 5 eps_svd.
CASES = [
    ("cube_p4_dense", wl.uniform_cube, 4000, 4, 32, 1, 0.0, 1e-9),
    ("gauss_p5_dense", wl.gaussian_mixture, 3000, 5, 16, 2, 0.0, 1e-9),
    ("cube_p6_k127", wl.uniform_cube, 4000, 6, 48, 1, 5e-7, 5 * 5e-7),
    ("sphere_p6_k116", wl.sphere_surface, 3000, 6, 24, 2, 1e-6, 5 * 1e-6),
]


@pytest.mark.parametrize("kind,gen,n,p,ncrit,nrhs,eps_svd,bar", CASES, ids=[c[0] for c in CASES])
def test_fp64_run_of_the_library_scheme_matches_the_oracle(kind, gen, n, p, ncrit, nrhs,
                                                           eps_svd, bar):
    x, q = gen(n, 33, nrhs=nrhs)
    P = FMMPlan(x, p, ncrit, host_only=1, eps_svd=eps_svd)
    phi, mid = run_fp64(P, x, q)
    K = ok.KIFMM(x, p, ncrit)
    ref = K.evaluate(q)
    errs = {"phi": rel(phi, ref)}
    keys, h, s, Uk = mid["keys"], mid["h"], mid["s"], mid["Uk"]
    k_up, k_dn = k1(AO * s, AI * s), k1(AI * s, AO * s)
    pairs = {"up": [], "down": [], "m2l": []}
    for b, r in enumerate(map(tuple, keys)):
        if r[0] < 2:
            continue
        pairs["up"].append((k_up @ mid["up"][b], k_up @ K.up[r]))
        pairs["down"].append((k_dn @ mid["down"][b], k_dn @ K.down[r]))
        if b in mid["chat"]:
            pairs["m2l"].append((Uk @ mid["chat"][b] / (4 * np.pi * h[b]), K.m2l_check[r]))
    for name, pr in pairs.items():
        got, want = np.concatenate([a for a, _ in pr]), np.concatenate([b for _, b in pr])
        errs[name] = rel(got, want)
    print(kind, "k", P.info("rank_m2l"), {a: f"{v:.1e}" for a, v in errs.items()})
    assert max(errs.values()) <= bar, errs
    assert len(pairs["m2l"]) == len(K.m2l_check)


@pytest.mark.parametrize("plant", ["l2l_child", "s_transpose"])
def test_the_comparison_sees_a_planted_mistake(plant):
    """The same comparison with one mistake planted in the FP64 run: the
    potentials must be off by far more than any bar above."""
    x, q = wl.uniform_cube(4000, 33)
    P = FMMPlan(x, 4, 32, host_only=1, eps_svd=0.0)
    ref = ok.KIFMM(x, 4, 32).evaluate(q)
    good, _ = run_fp64(P, x, q)
    bad, _ = run_fp64(P, x, q, plant=plant)
    assert rel(good, ref) <= 1e-9
    assert rel(bad, ref) >= 1e-3, rel(bad, ref)

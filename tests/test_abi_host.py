"""C-ABI host logic, no GPU needed: the library loads and exports every
declared symbol; host-only plans build the same octree, point partition and
U/V/W/X lists as the oracle (bit-exact: this is index work); the FP64
operators are consistent with the oracle's kernel matrices; invalid
arguments come back as status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import kifmm as ok
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "kifmm.h")).read()
    declared = set(re.findall(r"\b(fmm_[a-z_]+)\s*\(", header))
    assert declared == set(N.EXPORTS)
    lib = ctypes.CDLL(N.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def _plan_keys(P):
    keys = P.array("node_keys").reshape(-1, 4)
    return [tuple(int(v) for v in k) for k in keys]


def _csr(P, name, keys):
    ptr = P.array(name + "_ptr")
    idx = P.array(name + "_idx")
    out = {}
    for b in range(len(keys)):
        if ptr[b + 1] > ptr[b]:
            out[keys[b]] = sorted(keys[i] for i in idx[ptr[b]:ptr[b + 1]])
    return out


CASES = [("cube", 4000, 24, True), ("sphere", 3000, 8, True), ("gauss", 3000, 8, True),
         ("sphere", 3000, 8, False), ("gauss", 2500, 5, False)]


@pytest.mark.parametrize("kind,n,ncrit,balance", CASES)
def test_tree_and_lists_match_oracle(kind, n, ncrit, balance):
    gen = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface,
           "gauss": wl.gaussian_mixture}[kind]
    x, _ = gen(n, 31)
    P = FMMPlan(x, 4, ncrit, host_only=1, balance=int(balance))
    tree = ok.Octree(x, ncrit, balance=balance)
    U, V, W, X = ok.build_lists(tree)
    keys = _plan_keys(P)
    assert set(keys) == tree.nonempty
    assert len(keys) == len(set(keys))
    leaf = P.array("leaf_flag")
    assert {k for k, f in zip(keys, leaf) if f} == set(tree.leaves)
    # point partition: the sorted range of every box holds the oracle's points
    rng = P.array("node_range").reshape(-1, 2)
    perm = P.array("perm")
    assert np.array_equal(np.sort(perm), np.arange(n))
    for k, (a, b) in zip(keys, rng):
        assert np.array_equal(np.sort(perm[a:b]), np.sort(tree.points[k]))
    for name, ref in (("u", U), ("v", V), ("w", W), ("x", X)):
        got = _csr(P, name, keys)
        assert got == {k: sorted(v) for k, v in ref.items()}, name
    root = P.array("root")
    np.testing.assert_array_equal(root[:3], tree.centre)
    assert root[3] == tree.half_width


def test_counts_of_the_uniform_workload():
    x, _ = wl.uniform_cube(10_000, 0)
    P = FMMPlan(x, 4, 64, host_only=1)
    assert P.info("depth") == 3 and P.info("leaves") == 512 and P.info("nodes") == 585
    assert P.info("v_pairs") == 56_448
    assert P.info("w_pairs") == 0 and P.info("x_pairs") == 0
    assert P.info("nsurf") == 56


@pytest.mark.parametrize("p", [4, 6])
def test_operators_against_oracle_kernel(p):
    x, _ = wl.uniform_cube(500, 1)
    P = FMMPlan(x, p, 64, host_only=1)
    surf = P.array("surface").reshape(-1, 3)
    np.testing.assert_array_equal(surf, ok.surface_grid(p))
    k = P.info("rank_m2l")
    ns = len(surf)
    Uk = P.array("m2l_u").reshape(ns, k)
    Vk = P.array("m2l_v").reshape(ns, k)
    S = P.array("m2l_s").reshape(316, k, k)
    np.testing.assert_allclose(Uk.T @ Uk, np.eye(k), atol=1e-10)
    np.testing.assert_allclose(Vk.T @ Vk, np.eye(k), atol=1e-10)
    offs = [(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)
            if max(abs(a), abs(b), abs(c)) > 1]
    assert len(offs) == 316
    worst = 0.0
    for i, t in enumerate(offs):
        kt = 4 * np.pi * ok.laplace_kernel(1.05 * surf, 2.0 * np.array(t) + 1.05 * surf)
        err = np.linalg.norm(Uk @ S[i] @ Vk.T - kt) / np.linalg.norm(kt)
        worst = max(worst, err)
    assert worst < 50 * 1e-7, worst


def test_dense_m2l_option_keeps_full_rank():
    x, _ = wl.uniform_cube(300, 2)
    P = FMMPlan(x, 4, 32, host_only=1, eps_svd=0.0)
    assert P.info("rank_m2l") == 56
    S = P.array("m2l_s").reshape(316, 56, 56)
    surf = ok.surface_grid(4)
    kt = 4 * np.pi * ok.laplace_kernel(1.05 * surf, np.array([-3.0, -3.0, -3.0]) * 2 + 1.05 * surf)
    np.testing.assert_allclose(S[0], kt, rtol=1e-13)


def test_invalid_arguments():
    x, _ = wl.uniform_cube(10, 3)
    with pytest.raises(N.FMMError) as e:
        FMMPlan(x[:0], 4, 8, host_only=1)
    assert e.value.status == N.FMM_ERR_INVALID_ARG
    with pytest.raises(N.FMMError):
        FMMPlan(x, 1, 8, host_only=1)
    with pytest.raises(N.FMMError):
        FMMPlan(x, 4, 0, host_only=1)
    with pytest.raises(N.FMMError):
        FMMPlan(x, 4, 8, host_only=1, alpha_outer=3.0)
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(N.FMMError):
        FMMPlan(bad, 4, 8, host_only=1)
    L = N.lib()
    P = FMMPlan(x, 4, 8, host_only=1)
    with pytest.raises(N.FMMError):
        P.evaluate(np.ones(10, dtype=np.float32))
    L.fmm_destroy(None)
    # batch: no problems, an empty problem, a NULL source array
    h = ctypes.c_void_p()
    opts = N.Options()
    L.fmm_options_init(ctypes.byref(opts))
    opts.host_only = 1
    pts = np.ascontiguousarray(x)
    src = (ctypes.c_void_p * 2)(pts.ctypes.data, pts.ctypes.data)
    assert L.fmm_plan_create_batch_ex(src, None, (ctypes.c_int64 * 2)(10, 10), 0, 4, 8,
                                      ctypes.byref(opts), ctypes.byref(h)) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_create_batch_ex(src, None, (ctypes.c_int64 * 2)(10, 0), 2, 4, 8,
                                      ctypes.byref(opts), ctypes.byref(h)) == N.FMM_ERR_INVALID_ARG
    bad_src = (ctypes.c_void_p * 2)(pts.ctypes.data, None)
    assert L.fmm_plan_create_batch_ex(bad_src, None, (ctypes.c_int64 * 2)(10, 10), 2, 4, 8,
                                      ctypes.byref(opts), ctypes.byref(h)) == N.FMM_ERR_INVALID_ARG
    assert not h.value


def test_distinct_targets_build_the_tree_on_the_union():
    """Targets distinct from the sources: the octree and lists are the
    oracle's on the 2n points, sources keep their charge rows and targets
    get the potential rows."""
    x, _ = wl.uniform_cube(1500, 5)
    y, _ = wl.gaussian_mixture(1500, 6)
    n = len(x)
    P = FMMPlan(x, 4, 16, targets=y, host_only=1)
    assert P.info("n") == n and P.info("points") == 2 * n and P.info("problems") == 1
    u = np.vstack([x, y])
    tree = ok.Octree(u, 16)
    U, V, W, X = ok.build_lists(tree)
    keys = _plan_keys(P)
    assert set(keys) == tree.nonempty
    for name, ref in (("u", U), ("v", V), ("w", W), ("x", X)):
        assert _csr(P, name, keys) == {k: sorted(v) for k, v in ref.items()}, name
    perm = P.array("perm")
    qrow, orow = P.array("charge_row"), P.array("output_row")
    src = perm < n
    np.testing.assert_array_equal(qrow[src], perm[src])
    np.testing.assert_array_equal(orow[src], -1)
    np.testing.assert_array_equal(qrow[~src], -1)
    np.testing.assert_array_equal(orow[~src], perm[~src] - n)
    # targets given as the sources themselves: one point set
    Q = FMMPlan(x, 4, 16, targets=x, host_only=1)
    assert Q.info("points") == n
    np.testing.assert_array_equal(Q.array("charge_row"), Q.array("perm"))
    np.testing.assert_array_equal(Q.array("output_row"), Q.array("perm"))


def _batch_sets():
    sizes = [700, 37, 2500, 1, 1200]
    gens = [wl.uniform_cube, wl.sphere_surface, wl.gaussian_mixture, wl.uniform_cube,
            wl.sphere_surface]
    return [g(n, 40 + i)[0] for i, (g, n) in enumerate(zip(gens, sizes))]


def test_batch_plan_is_the_forest_of_single_plans():
    """A batch plan holds every problem's own tree and lists, renumbered: the
    boxes of problem i, in plan order, are the boxes of the single plan of
    problem i, and every list maps across."""
    sets = _batch_sets()
    targets = [None, None, wl.uniform_cube(2500, 9)[0], None, None]
    B = FMMPlan.batch(sets, 4, 20, target_sets=targets, host_only=1)
    sizes = [len(x) for x in sets]
    assert B.info("problems") == len(sets) and B.info("n") == sum(sizes)
    assert B.info("points") == sum(sizes) + 2500
    keys = B.array("node_keys").reshape(-1, 4)
    assert np.all(np.diff(keys[:, 0]) >= 0)  # level-major
    owner = B.array("node_problem")
    rng = B.array("node_range").reshape(-1, 2)
    perm, qrow, orow = B.array("perm"), B.array("charge_row"), B.array("output_row")
    roots = B.array("root").reshape(-1, 4)
    lists = {nm: (B.array(nm + "_ptr"), B.array(nm + "_idx")) for nm in "uvwx"}
    pt_base = row_base = 0
    pairs = {"p2p_pairs": 0, "v_pairs": 0, "u_pairs": 0, "surf_pairs": 0}
    for i, x in enumerate(sets):
        S = FMMPlan(x, 4, 20, targets=targets[i], host_only=1)
        ids = np.nonzero(owner == i)[0]
        np.testing.assert_array_equal(keys[ids], S.array("node_keys").reshape(-1, 4))
        np.testing.assert_array_equal(rng[ids], S.array("node_range").reshape(-1, 2) + pt_base)
        npts = S.info("points")
        sl = slice(pt_base, pt_base + npts)
        np.testing.assert_array_equal(perm[sl], S.array("perm") + pt_base)
        for got, ref in ((qrow[sl], S.array("charge_row")), (orow[sl], S.array("output_row"))):
            np.testing.assert_array_equal(got, np.where(ref >= 0, ref + row_base, -1))
        np.testing.assert_array_equal(roots[i], S.array("root"))
        for nm, (bptr, bidx) in lists.items():
            sptr, sidx = S.array(nm + "_ptr"), S.array(nm + "_idx")
            for b, gb in enumerate(ids):
                np.testing.assert_array_equal(bidx[bptr[gb]:bptr[gb + 1]],
                                              ids[sidx[sptr[b]:sptr[b + 1]]])
        for k in pairs:
            pairs[k] += S.info(k)
        pt_base += npts
        row_base += len(x)
    for k, v in pairs.items():
        assert B.info(k) == v, k


def test_single_point_and_duplicates():
    P = FMMPlan(np.array([[0.3, 0.2, 0.1]]), 4, 1, host_only=1)
    assert P.info("nodes") == 1 and P.info("leaves") == 1 and P.info("depth") == 0
    x = np.zeros((40, 3))
    P = FMMPlan(x, 4, 8, host_only=1, max_level=5)
    assert P.info("depth") == 5


def test_gradient_entry_point_arguments():
    """fmm_evaluate_gradient refuses NULL gradients and host-only plans with
    status codes (no GPU needed)."""
    x, q = wl.uniform_cube(200, 4)
    P = FMMPlan(x, 4, 32, host_only=1)
    L = N.lib()
    qf = np.ascontiguousarray(q[:, 0], dtype=np.float32)
    g = np.zeros((len(x), 1, 3))
    phi = np.zeros((len(x), 1))
    assert L.fmm_evaluate_gradient(P._h, qf.ctypes.data, 1, phi.ctypes.data, None,
                                   None) == N.FMM_ERR_INVALID_ARG
    assert "gradients" in N.lib().fmm_last_error().decode()
    assert L.fmm_evaluate_gradient(P._h, qf.ctypes.data, 1, None, g.ctypes.data,
                                   None) == N.FMM_ERR_INVALID_ARG
    assert "host-only" in N.lib().fmm_last_error().decode()
    assert L.fmm_evaluate_gradient(None, qf.ctypes.data, 1, None, g.ctypes.data,
                                   None) == N.FMM_ERR_INVALID_ARG


def test_failure_hook_option_values():
    """FMM_OPT_TEST_M2L_STALL takes 0 or 1 and nothing else (no GPU needed;
    the stall itself is exercised in test_gpu_failure.py)."""
    x, _ = wl.uniform_cube(200, 5)
    P = FMMPlan(x, 4, 32, host_only=1)
    L = N.lib()
    assert L.fmm_plan_set_option(P._h, N.OPT_TEST_M2L_STALL, 1.0) == N.FMM_OK
    assert L.fmm_plan_set_option(P._h, N.OPT_TEST_M2L_STALL, 0.0) == N.FMM_OK
    assert L.fmm_plan_set_option(P._h, N.OPT_TEST_M2L_STALL, 2.0) == N.FMM_ERR_INVALID_ARG
    assert "0 or 1" in L.fmm_last_error().decode()


def test_workspace_export_needs_an_evaluation():
    """fmm_plan_get_workspace refuses host-only plans, plans never evaluated
    and unknown arrays (no GPU needed)."""
    x, _ = wl.uniform_cube(200, 6)
    P = FMMPlan(x, 4, 32, host_only=1)
    need = ctypes.c_int64()
    L = N.lib()
    assert L.fmm_plan_get_workspace(P._h, 0, None, 0, ctypes.byref(need)) == N.FMM_ERR_INVALID_ARG
    assert "no evaluation" in L.fmm_last_error().decode()
    assert L.fmm_plan_get_workspace(None, 0, None, 0, None) == N.FMM_ERR_INVALID_ARG


def test_python_constants_match_the_header():
    """Every info key, array id, option key, workspace id, status and M2L mode
    the header declares has the same value in the Python binding, and the
    binding names no key the header lacks."""
    header = open(os.path.join(ROOT, "include", "kifmm.h")).read()

    def enum(prefix):
        return {m.group(1).lower(): int(m.group(2))
                for m in re.finditer(r"\b" + prefix + r"([A-Z0-9_]+)\s*=\s*(\d+)", header)}

    assert enum("FMM_INFO_") == N.INFO
    assert enum("FMM_ARRAY_") == {k: v[0] for k, v in N.ARRAYS.items()}
    for name, value in enum("FMM_OPT_").items():
        assert getattr(N, "OPT_" + name.upper()) == value, name
    for name, value in enum("FMM_ERR_").items():
        assert getattr(N, "FMM_ERR_" + name.upper()) == value, name
    for name, value in enum("FMM_M2L_").items():
        assert getattr(N, "M2L_" + name.upper()) == value, name
    for name, value in enum("FMM_TREE_").items():
        assert getattr(N, "TREE_" + name.upper()) == value, name
    assert enum("FMM_WORK_") == {"up": 0, "down": 1, "qhat": 2, "chat": 3}
    assert N.FMM_OK == 0


@pytest.mark.parametrize("label,kw,fragment", [
    ("+inf", {"inf": np.inf}, "non-finite"), ("-inf", {"inf": -np.inf}, "non-finite"),
    ("nan target", {"nan_target": True}, "non-finite"),
    ("p = 11", {"p": 11}, "p must be in [2, 10]"),
    ("max_level 17", {"max_level": 17}, "max_level"), ("max_level -1", {"max_level": -1}, "max_level"),
    ("radii swapped", {"alpha_inner": 2.95, "alpha_outer": 1.05}, "alpha_inner"),
    ("alpha_inner <= 1", {"alpha_inner": 0.5}, "alpha_inner"),
    ("rcond < 0", {"rcond": -1.0}, "rcond"), ("eps_svd < 0", {"eps_svd": -1.0}, "eps_svd"),
    ("eps_svd nan", {"eps_svd": float("nan")}, "eps_svd"),
])
def test_invalid_plan_arguments_are_refused_with_a_message(label, kw, fragment):
    x, _ = wl.uniform_cube(50, 3)
    kw = dict(kw)
    p = kw.pop("p", 4)
    targets = None
    if "inf" in kw:
        x = x.copy()
        x[2, 0] = kw.pop("inf")
    if kw.pop("nan_target", False):
        targets = x.copy()
        targets[1, 2] = np.nan
    with pytest.raises(N.FMMError) as e:
        FMMPlan(x, p, 8, targets=targets, host_only=1, **kw)
    assert e.value.status == N.FMM_ERR_INVALID_ARG
    assert fragment in str(e.value), (label, str(e.value))


def test_null_and_negative_arguments():
    x, _ = wl.uniform_cube(50, 3)
    pts = np.ascontiguousarray(x)
    L = N.lib()
    h = ctypes.c_void_p()
    assert L.fmm_plan_create(None, None, 10, 4, 8, ctypes.byref(h)) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_create(pts.ctypes.data, None, 50, 4, 8, None) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_create(pts.ctypes.data, None, -5, 4, 8, ctypes.byref(h)) == N.FMM_ERR_INVALID_ARG
    assert not h.value
    P = FMMPlan(x, 4, 8, host_only=1)
    assert L.fmm_plan_info(P._h, 0, None) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_set_option(P._h, 99, 1.0) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_set_option(P._h, N.OPT_M2L_MODE, 7.0) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_set_option(P._h, N.OPT_GEMM_SHAPE, 5.0) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_set_option(P._h, N.OPT_FORCE_KNOBS, 4.0) == N.FMM_ERR_INVALID_ARG
    assert L.fmm_plan_set_option(P._h, N.OPT_FORCE_KNOBS, 0.5) == N.FMM_ERR_INVALID_ARG
    for v in (-1.0, 0.0, 3.0):
        assert L.fmm_plan_set_option(P._h, N.OPT_FORCE_KNOBS, v) == 0


def test_surface_and_direct_pair_counts():
    """FMM_INFO_SURF_PAIRS and FMM_INFO_WX_DIRECT_PAIRS count the leaf pass's
    pairs beside the near field.  For every leaf B: its points times the
    surface points of its own downward equivalent surface (levels >= 2) and
    of each W box's upward surface, except that (direct_wx, the default) a
    W box that is a leaf with no more points than a surface contributes
    points x points, and so does every X(B) leaf when B itself has no more
    points than a surface; without direct_wx every W box is a surface."""
    x, _ = wl.gaussian_mixture(6000, 3)
    for p in (3, 5):
        ns = 6 * (p - 1) ** 2 + 2
        for direct in (1, 0):
            P = FMMPlan(x, p, 24, host_only=1, direct_wx=direct)
            keys = P.array("node_keys").reshape(-1, 4)
            rng = P.array("node_range").reshape(-1, 2)
            leaf = P.array("leaf_flag") > 0
            wptr, widx = P.array("w_ptr"), P.array("w_idx")
            xptr, xidx = P.array("x_ptr"), P.array("x_idx")
            npts = rng[:, 1] - rng[:, 0]
            assert P.info("nsurf") == ns

            def small(a):
                return direct and leaf[a] and npts[a] <= ns
            surf = pairs = 0
            for b in np.nonzero(leaf)[0]:
                nsurf = int(keys[b, 0] >= 2)
                for a in widx[wptr[b]:wptr[b + 1]]:
                    if small(a):
                        pairs += int(npts[b] * npts[a])
                    else:
                        nsurf += 1
                if small(b):
                    pairs += int(npts[b] * npts[xidx[xptr[b]:xptr[b + 1]]].sum())
                surf += int(npts[b]) * nsurf * ns
            assert np.count_nonzero(np.diff(wptr)[leaf]) > 0  # W lists present
            assert P.info("surf_pairs") == surf
            assert P.info("wx_direct_pairs") == pairs
            assert (pairs > 0) == bool(direct)

"""The seeded input generators against the input recipe they state (no GPU):
ranges, distributions, independence of seeds and the named workloads'
parameters.  Statistical checks use enough points that their bounds sit many
standard errors away from the expected values."""
import numpy as np
import pytest

from paper_2303_08394_gb300 import workloads as wl

N = 200_000


def test_uniform_cube():
    x, q = wl.uniform_cube(N, 3, nrhs=2)
    assert x.shape == (N, 3) and q.shape == (N, 2)
    assert x.dtype == np.float64 and q.dtype == np.float64
    assert x.min() >= 0.0 and x.max() < 1.0
    assert q.min() >= -1.0 and q.max() <= 1.0
    np.testing.assert_allclose(x.mean(0), 0.5, atol=0.005)           # se 6.5e-4
    np.testing.assert_allclose(x.var(0), 1 / 12, rtol=0.02)
    np.testing.assert_allclose(q.mean(0), 0.0, atol=0.01)
    np.testing.assert_allclose(q.var(0), 1 / 3, rtol=0.02)
    assert abs(np.corrcoef(q[:, 0], q[:, 1])[0, 1]) < 0.01            # independent columns


def test_sphere_surface():
    x, q = wl.sphere_surface(N, 4)
    np.testing.assert_allclose(np.linalg.norm(x, axis=1), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(x.mean(0), 0.0, atol=0.01)             # uniform on the sphere
    np.testing.assert_allclose((x ** 2).mean(0), 1 / 3, rtol=0.02)
    # uniform on the sphere: z is uniform in [-1, 1]
    hist, _ = np.histogram(x[:, 2], bins=10, range=(-1, 1))
    np.testing.assert_allclose(hist / N, 0.1, atol=0.005)
    np.testing.assert_allclose(q.mean(), 0.0, atol=0.01)
    np.testing.assert_allclose(q.std(), 1.0, rtol=0.01)


def test_gaussian_mixture():
    sigma = 0.05
    x, q = wl.gaussian_mixture(N, 5, sigma=sigma)
    assert x.shape == (N, 3)
    # the centres are the first 8 x 3 draws of the stream (the recipe's
    # order: centres, then assignments, then offsets)
    centres = np.random.default_rng(5).random((8, 3))
    d = np.min(np.linalg.norm(x[:, None, :] - centres[None, :, :], axis=2), axis=1)
    # |offset| / sigma is chi-distributed with 3 degrees of freedom (median
    # 1.538); the nearest centre can only be nearer than the drawn one
    med = np.median(d) / sigma
    assert 1.40 < med < 1.56, med
    assert np.quantile(d, 0.999) / sigma < 5.0
    assert (x < 0).any() or (x > 1).any()                              # not clipped
    assert q.min() >= -1.0 and q.max() <= 1.0


def test_seeds_reproduce_and_differ():
    for gen in (wl.uniform_cube, wl.sphere_surface, wl.gaussian_mixture):
        a, qa = gen(1000, 11)
        b, qb = gen(1000, 11)
        c, _ = gen(1000, 12)
        assert np.array_equal(a, b) and np.array_equal(qa, qb)
        assert not np.array_equal(a, c)
        # the points do not depend on nrhs: they are drawn before the charges
        d, qd = gen(1000, 11, nrhs=3)
        assert np.array_equal(a, d) and qd.shape == (1000, 3)


def test_problem_sizes_and_batches():
    sizes = wl.log_uniform_sizes(20_000, 6)
    assert sizes.min() >= 1000 and sizes.max() <= 100_000
    np.testing.assert_allclose(np.log10(sizes).mean(), 4.0, atol=0.02)
    hist, _ = np.histogram(np.log10(sizes), bins=4, range=(3, 5))
    np.testing.assert_allclose(hist / len(sizes), 0.25, atol=0.02)
    probs = wl.batch_problems(6, 7)
    assert [len(x) for x, _ in probs] == list(wl.log_uniform_sizes(6, 7))
    assert len({x[0, 0] for x, _ in probs}) == 6                       # independent streams


def test_sample_targets():
    idx = wl.sample_targets(10_000, 1000, 0)
    assert len(idx) == 1000 and len(np.unique(idx)) == 1000
    assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < 10_000
    assert np.array_equal(idx, wl.sample_targets(10_000, 1000, 0))
    assert len(wl.sample_targets(50, 1000, 0)) == 50


@pytest.mark.parametrize("name,kind,n,p,ncrit,nrhs", [
    ("cube_n1e4_p4_ncrit64", "cube", 10_000, 4, 64, 1),
    ("cube_n1e6_p6_ncrit150", "cube", 1_000_000, 6, 150, 1),
    ("sphere_n4e6_p7_ncrit128", "sphere", 4_000_000, 7, 128, 1),
    ("cube_n1e6_p6_ncrit150_nrhs64", "cube", 1_000_000, 6, 150, 64),
    ("gauss8_n1.6e7_p8_ncrit128_nrhs8", "gauss", 16_000_000, 8, 128, 8),
    ("batch256_cube_p6_ncrit150", "batch", 6_523_380, 6, 150, 1),
])
def test_named_workloads(name, kind, n, p, ncrit, nrhs):
    w = wl.WORKLOADS[name]
    assert (w.name, w.kind, w.n, w.p, w.ncrit, w.nrhs) == (name, kind, n, p, ncrit, nrhs)


def test_batch_workload_is_the_concatenated_problems():
    w = wl.WORKLOADS["batch256_cube_p6_ncrit150"]
    sets = w.problem_sets(0)
    assert len(sets) == 256 and w.problems == 256
    x, q = w.generate(0)
    assert len(x) == w.n == sum(len(a) for a, _ in sets)
    np.testing.assert_array_equal(x[:len(sets[0][0])], sets[0][0])
    np.testing.assert_array_equal(q[-len(sets[-1][1]):], sets[-1][1])

"""CPU checks of the seeded input generators against their stated recipes:
the SplitMix64 stream against the generator's published first outputs,
uniforms and Box-Muller normals by their moments, subset regeneration,
per-dimension scales and LogNormal row norms, the clustered-user mixture,
distinct ids and the workload shapes (Table I)."""
import numpy as np
import pytest

from paper_1706_01449_gb300 import synth


def test_splitmix64_first_outputs_for_seed_zero():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the counter's i-th
    # value is i * golden, so mix(i * golden) are the generator's outputs
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        ctr = np.arange(3, dtype=np.uint64) * g
    out = synth._splitmix64(ctr)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_moments():
    u = synth.uniform(1, 2, 400000)
    assert (u > 0).all() and (u < 1).all()
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = synth.normal(1, 3, 400000)
    assert abs(z.mean()) < 6e-3 and abs(z.var() - 1) < 1e-2
    assert abs((z ** 4).mean() - 3) < 0.06  # kurtosis of a normal


@pytest.mark.parametrize("offset,n", [(0, 10), (7, 13), (1000, 1)])
def test_streams_regenerate_any_subset(offset, n):
    full_u = synth.uniform(5, 9, 2000)
    np.testing.assert_array_equal(synth.uniform(5, 9, n, offset), full_u[offset:offset + n])
    full_z = synth.normal(5, 9, 2000)
    np.testing.assert_array_equal(synth.normal(5, 9, n, offset), full_z[offset:offset + n])


def test_streams_differ_by_seed_and_stream():
    a = synth.uniform(0, 1, 100)
    assert not np.array_equal(a, synth.uniform(1, 1, 100))
    assert not np.array_equal(a, synth.uniform(0, 2, 100))
    np.testing.assert_array_equal(a, synth.uniform(0, 1, 100))


def test_gaussian_rows_scales_and_lognormal_norms():
    n, f = 60000, 12
    x = synth.gaussian_rows(n, f, 4, synth.S_ITEMS).astype(np.float64)
    sd = x.std(axis=0)
    np.testing.assert_allclose(sd, 1 / np.sqrt(np.arange(1, f + 1)), rtol=0.02)
    y = synth.gaussian_rows(n, f, 4, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.1, 0.7)).astype(np.float64)
    ln = np.log(np.linalg.norm(y, axis=1))
    assert abs(ln.mean() - 0.1) < 0.01 and abs(ln.std() - 0.7) < 0.01
    # rescaling keeps each row's direction
    cos = (x * y).sum(1) / (np.linalg.norm(x, axis=1) * np.linalg.norm(y, axis=1))
    assert (cos > 1 - 1e-6).all()
    # chunked generation equals one piece
    np.testing.assert_array_equal(synth.gaussian_rows(1000, f, 4, synth.S_ITEMS, chunk=37 * f),
                                  synth.gaussian_rows(1000, f, 4, synth.S_ITEMS))


def test_clustered_users_mixture():
    n, f, nd = 20000, 16, 32
    U = synth.clustered_users(n, f, 2, n_dirs=nd, noise=0.2).astype(np.float64)
    ln = np.log(np.linalg.norm(U, axis=1))
    assert abs(ln.mean()) < 0.01 and abs(ln.std() - 0.3) < 0.01
    dirs = synth.normal(2, synth.S_DIRS, nd * f).reshape(nd, f)
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    cos = (U / np.linalg.norm(U, axis=1)[:, None]) @ dirs.T
    best = cos.max(axis=1)
    # direction + 0.2 N(0, I) noise: cos ~ 1 / sqrt(1 + 0.04 f) = 0.78 at f = 16
    assert abs(np.median(best) - 1 / np.sqrt(1 + 0.04 * f)) < 0.05
    # uneven clusters: LogNormal(0, 1) weights
    counts = np.bincount(cos.argmax(axis=1), minlength=nd)
    assert counts.max() > 3 * max(1, np.median(counts))


def test_distinct_ids_and_workload_shapes():
    ids = synth.distinct_ids(1000, 300, 3, synth.S_INIT)
    assert len(set(ids.tolist())) == 300 and ids.min() >= 0 and ids.max() < 1000
    with pytest.raises(ValueError):
        synth.distinct_ids(5, 6, 0, 1)
    W = synth.WORKLOADS
    assert (W["netflix-480189x17770"]["n_users"], W["netflix-480189x17770"]["n_items"]) == (480189, 17770)
    assert (W["kdd-1000000x624961"]["n_users"], W["kdd-1000000x624961"]["n_items"]) == (1000000, 624961)
    assert (W["r2-1823179x136736"]["n_users"], W["r2-1823179x136736"]["n_items"]) == (1823179, 136736)
    assert synth.make_users(W["small-2048x1024-f32"], 0).shape == (2048, 32)
    s = synth.serving_users(50, 128, 1)
    assert s.shape == (50, 128) and abs(s.std() * np.sqrt(128) - 1) < 0.05

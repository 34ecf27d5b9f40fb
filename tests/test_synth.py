"""The seeded input generators (synth/), which both sides of every parity
test read: deterministic per seed, unit-normalised, drawn from the stated
mixture, and the workloads' shapes as documented."""
import numpy as np
import pytest

import synth


def test_draws_are_deterministic_and_seed_dependent():
    mix = synth.Mixture(12, 5, "anisotropic", param_seed=3, mean_scale=0.2)
    a, b, c = mix.sample(500, 7), mix.sample(500, 7), mix.sample(500, 8)
    assert a.dtype == np.float32 and a.shape == (500, 12)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    again = synth.Mixture(12, 5, "anisotropic", param_seed=3, mean_scale=0.2)
    np.testing.assert_array_equal(again.sample(500, 7), a)      # parameters fixed by param_seed


@pytest.mark.parametrize("kind", ["isotropic", "anisotropic"])
def test_draws_are_unit_vectors(kind):
    X = synth.Mixture(16, 4, kind, 0.3, param_seed=5).sample(3000, 9)
    np.testing.assert_allclose(np.linalg.norm(X.astype(np.float64), axis=1), 1.0, atol=1e-6)


def test_isotropic_draws_cluster_around_their_component_means():
    # sigma small against the spread of the means: every draw's nearest
    # normalised mean is the component it came from, and all components occur
    mix = synth.Mixture(32, 6, "isotropic", 0.05, param_seed=11)
    X = mix.sample(2000, 12)
    mu = mix.means / np.linalg.norm(mix.means, axis=1, keepdims=True)
    nearest = np.argmax(X @ mu.T, axis=1)
    rng = np.random.default_rng(12)
    comp = rng.integers(0, 6, size=2000)                         # the sampler's first draw
    np.testing.assert_array_equal(nearest, comp)
    assert set(np.unique(comp)) == set(range(6))


def test_anisotropic_factors_are_rotations_times_the_spectrum():
    mix = synth.Mixture(10, 3, "anisotropic", param_seed=13)
    for f in mix.factors:
        ev = np.linalg.eigvalsh(f @ f.T)                          # U diag(e) U^T
        assert ev.min() >= 0.01 - 1e-9 and ev.max() <= 1.0 + 1e-9


def test_a_draw_of_whole_chunks_is_a_prefix():
    mix = synth.Mixture(4, 3, "isotropic", 0.3, param_seed=1)
    a = mix.sample(2 * 64, 5, chunk=64)
    b = mix.sample(3 * 64 + 17, 5, chunk=64)
    np.testing.assert_array_equal(a, b[:128])


def test_init_indices_distinct_sorted_and_bounded():
    idx = synth.init_indices(1000, 64, 3)
    assert idx.dtype == np.int32 and len(np.unique(idx)) == 64
    assert np.all(np.diff(idx) > 0) and idx.min() >= 0 and idx.max() < 1000
    np.testing.assert_array_equal(idx, synth.init_indices(1000, 64, 3))
    with pytest.raises(ValueError):
        synth.init_indices(10, 11, 0)


def test_poisson_arrivals_have_the_rate():
    t = synth.poisson_arrivals(1000.0, 20_000, seed=4)
    assert np.all(np.diff(t) > 0)
    assert 20_000 / t[-1] == pytest.approx(1000.0, rel=0.03)


def test_request_mix_ranges():
    k, t = synth.request_mix(5000, seed=6)
    assert set(np.unique(k)) == {10, 100}
    assert t.min() >= 32 and t.max() <= 512 and t.dtype == np.int32


def test_workload_shapes_as_documented():
    w = synth.WORKLOADS
    assert (w["glove"].n, w["glove"].d, w["glove"].c, w["glove"].components) == (1_183_514, 100, 2000, 500)
    assert (w["precision"].n, w["precision"].d, w["precision"].c) == (10_000_000, 96, 10_000)
    assert (w["serving"].n, w["serving"].d, w["serving"].c) == (100_000_000, 128, 40_000)
    assert (w["multilevel"].n, w["multilevel"].c) == (10_000_000, 100_000)
    X, Q, init = synth.workload_arrays("tiny", n=3000, nq=50)
    assert X.shape == (3000, 64) and Q.shape == (50, 64) and len(init) == 64

"""The seeded input recipes: determinism, ranges and the properties the stored workloads rely on."""
import numpy as np

from paper_2601_11437_gb300 import inputs


def test_streams_are_deterministic_and_in_range():
    a = inputs.uniform_locations(1000, 11)
    assert np.array_equal(a, inputs.uniform_locations(1000, 11))
    assert a.shape == (1000, 2) and a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, inputs.uniform_locations(1000, 12))
    e = inputs.standard_normal(100001, 3)
    assert abs(e.mean()) < 0.01 and abs(e.std() - 1.0) < 0.01


def test_splitmix64_known_answers():
    # SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) from state 0: the first three outputs of the
    # published generator, which advances the state by 0x9E3779B97F4A7C15 before each output
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        states = np.array([g * np.uint64(k) for k in (1, 2, 3)], dtype=np.uint64)
    assert [int(v) for v in inputs._mix64(states)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                       0x06C45D188009454F]
    # a stream is the generator started from the mixed (seed, stream) key
    key = int(inputs._mix64(np.array([(5 << 32) | 2], dtype=np.uint64))[0])
    with np.errstate(over="ignore"):
        first = inputs._mix64(np.array([np.uint64(key) + g], dtype=np.uint64))[0]
    assert inputs.random_u64(5, 2, 3)[0] == first


def test_batched_recipe_is_a_prefix_of_the_larger_one():
    # the stored 256-field workload is the first 256 fields of the 2,048-field recipe
    small, large = inputs.batched_fields(256), inputs.batched_fields(2048)
    assert small == large[:256]
    ns = np.array([f.n for f in large])
    assert ns.min() >= 256 and ns.max() <= 4096
    th = np.array([f.theta_true for f in large])
    assert (th[:, 0] >= 0.5).all() and (th[:, 0] <= 2.0).all()
    assert (th[:, 1] >= 0.02).all() and (th[:, 1] <= 0.3).all()
    assert (th[:, 2] >= 0.3).all() and (th[:, 2] <= 2.5).all()


def test_simulation_study_seeds_are_distinct():
    # Sec. 3: five settings x three sizes; realisations share the design of their size
    assert len(inputs.SIM_SETTINGS) == 5 and inputs.SIM_SIZES == (1600, 3600, 6400)
    seen = set()
    for si in range(len(inputs.SIM_SETTINGS)):
        for n in inputs.SIM_SIZES:
            for r in range(50):
                key = inputs.SIM_SEED * 100_000_000 + si * 1_000_000 + n * 100 + r
                assert key < 2 ** 32 and key not in seen
                seen.add(key)
    e0 = inputs.sim_normals(0, 1600, 0)
    assert not np.array_equal(e0, inputs.sim_normals(0, 1600, 1))
    assert not np.array_equal(e0, inputs.sim_normals(1, 1600, 0))
    assert np.array_equal(inputs.sim_locations(1600), inputs.sim_locations(1600))

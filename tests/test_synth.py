"""The seeded input generator makes valid, balanced APRs of the intended sparsity (CPU only)."""
import numpy as np
import pytest

import aprsynth as S


@pytest.mark.parametrize("seed", range(4))
def test_random_balanced_apr_is_a_balanced_partition(seed):
    apr = S.random_balanced_apr((12, 16, 10), 1, seed=seed)
    S.validate_apr(apr, check_balance=True)


def test_blob64_workload_shape():
    apr = S.make_config("blob64", use_cache=False)
    S.validate_apr(apr, check_balance=True)
    frac = apr.n_particles / np.prod(apr.dims)
    assert 0.05 <= frac <= 0.10, frac           # ~5-10% particles
    assert apr.l_max == 6
    assert np.all(apr.values > 0)


def test_generator_is_deterministic():
    a = S.make_config("blob64", use_cache=False)
    b = S.make_config("blob64", use_cache=False)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.y_idx, b.y_idx)
    assert np.array_equal(a.values, b.values)


def test_uniform_and_hand_built():
    a = S.uniform_level_apr((8, 8, 8), 2)
    assert a.n_particles == 64 and a.l_max == 3
    S.validate_apr(a)
    b = S.apr_from_particles((2, 2, 2), 1, [(1, z, x, y, 1.0) for z in range(2) for x in range(2) for y in range(2)])
    assert b.n_particles == 8

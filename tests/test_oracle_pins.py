"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin, oracle_lib):
    err, tol = pin(oracle_lib)
    assert err <= tol, f"{pin.__name__}: error {err:.3e} > tolerance {tol:.3e}"


def test_knot_golden_values_are_a_partition_of_unity():
    for t, B in P.load_knots():
        assert abs(B.sum() - 1.0) < 1e-15


def test_oracle_threads_deterministic(oracle_lib):
    """The dense adjoint depends only on the thread count; forward is per-voxel."""
    import numpy as np
    import oracle

    rng = np.random.default_rng(3)
    shape, spacing = (13, 9, 10), (3, 2, 4)
    G = rng.normal(size=shape + (3,))
    a1 = oracle.adjoint(G, spacing, nthreads=1)
    a4 = oracle.adjoint(G, spacing, nthreads=4)
    assert np.max(np.abs(a1 - a4)) < 1e-12
    phi = rng.uniform(-1, 1, oracle.grid_shape(shape, spacing) + (3,))
    assert np.array_equal(oracle.forward(phi, shape, spacing, nthreads=1),
                          oracle.forward(phi, shape, spacing, nthreads=3))


def test_oracle_empty_volume(oracle_lib):
    import numpy as np
    import oracle

    phi = np.ones(oracle.grid_shape((0, 4, 4), (2, 2, 2)) + (3,))
    assert oracle.forward(phi, (0, 4, 4), (2, 2, 2)).shape == (0, 4, 4, 3)
    d = oracle.adjoint(np.zeros((0, 4, 4, 3)), (2, 2, 2))
    assert d.shape == (3, 5, 5, 3) and not d.any()

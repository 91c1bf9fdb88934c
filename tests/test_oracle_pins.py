"""The FP64 oracle against its pins (CPU only)."""
import pytest

from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin, oracle_lib):
    pin(oracle_lib)


def test_oracle_rejects_bad_arguments():
    import numpy as np
    import oracle
    x = np.zeros((5, 2, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.msd(x, 5, 1)          # tau_max > T-1
    with pytest.raises(ValueError):
        oracle.acf(x, 2, 0)          # stride < 1
    with pytest.raises(ValueError):
        oracle.einstein(np.arange(10.0), 1.0, 3, 5, 5)


def test_oracle_thread_count_does_not_change_bits():
    import numpy as np
    import oracle
    rng = np.random.default_rng(3)
    x = rng.normal(size=(60, 300, 3)).astype(np.float32)
    a = oracle.msd(x, 59, 1, nthreads=1)
    b = oracle.msd(x, 59, 1, nthreads=7)
    assert np.array_equal(a, b)

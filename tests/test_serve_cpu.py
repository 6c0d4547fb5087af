"""Host logic of the server that needs no GPU: memory-budget admission and
Poisson arrivals."""
import numpy as np
import pytest

from paper_2402_01296_gb300 import serve


def test_memory_budget_admission():
    b = serve.MemoryBudget(100)
    assert b.reserve(60) and not b.reserve(41) and b.reserve(40)
    b.release(60)
    assert b.used == 40 and b.reserve(60) and not b.reserve(1)
    with pytest.raises(AssertionError):
        b.release(101)


def test_poisson_arrivals_rate():
    t = serve.poisson_arrivals(500.0, 20.0, seed=3)
    assert np.all(np.diff(t) > 0) and t[-1] <= 20.0
    assert abs(len(t) / 20.0 - 500.0) < 5 * np.sqrt(500.0 / 20.0)  # within 5 sigma of the rate

"""Host-side helpers of the drift study (no GPU): the power-law fit that reads
the growth exponent of the centre-of-mass displacement, and the relative
total force |sum m a| / sum m |a|."""
import numpy as np

from paper_2502_01496_gb300 import drift


def test_fit_power_recovers_exponent_and_prefactor():
    t = np.linspace(0.01, 2.0, 50)
    for p, c in ((1.5, 3e-7), (2.0, 0.25)):
        fp, fc = drift._fit_power(t, c * t ** p)
        assert abs(fp - p) < 1e-10 and abs(fc / c - 1.0) < 1e-10


def test_fit_power_ignores_non_positive_samples_and_needs_three():
    t = np.array([0.0, 1.0, 2.0, 4.0])
    y = np.array([0.0, 1.0, 4.0, 16.0])
    p, c = drift._fit_power(t, y)
    assert abs(p - 2.0) < 1e-12 and abs(c - 1.0) < 1e-12
    assert drift._fit_power(np.array([1.0, 2.0]), np.array([1.0, 2.0])) == (None, None)


def test_relative_total_force():
    rng = np.random.default_rng(3)
    m = rng.uniform(0.5, 2.0, 64)
    a = rng.normal(size=(64, 3))
    # equal and opposite pairs: the total force vanishes
    m2 = np.concatenate([m, m])
    a2 = np.concatenate([a / m[:, None], -a / m[:, None]])
    assert drift._rel_force(m2, a2) < 1e-15
    # all forces parallel: the ratio is one
    a3 = np.tile([0.0, 0.0, 1.0], (64, 1))
    assert abs(drift._rel_force(m, a3) - 1.0) < 1e-15

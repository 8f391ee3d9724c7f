"""Host-side post-processing of the Hopf study (Sec. 4.4.2) in bench.py, on
signals whose answers are known in closed form."""
import numpy as np

import bench


def test_energy_of_a_sinusoid():
    # E_u^2 = (L / u0) var(u); var of A sin + c over whole periods is A^2 / 2
    L, u0, A = 99.0, 0.1, 3e-3
    t = np.arange(4000)
    u = 0.02 + A * np.sin(2 * np.pi * t / 400)
    np.testing.assert_allclose(bench.hopf_energy(u, L, u0), (L / u0) * A * A / 2, rtol=1e-12)
    assert bench.hopf_energy(np.full(100, 0.3), L, u0) == 0.0


def test_line_fit_finds_the_critical_reynolds_number():
    res = np.array([6800, 7000, 7200, 7400, 7600, 7800])
    e2 = np.where(res > 7135, 2e-5 * (res - 7135), 1e-9)  # steady below Re_c, linear above
    assert abs(bench.hopf_fit(res, e2) - 7135) < 1e-6
    assert bench.hopf_fit(res, np.zeros(6)) is None


def test_dominant_frequency_in_convective_units():
    L, u0 = 99.0, 0.1
    steps_per_unit = L / u0  # 990 steps per non-dimensional time unit
    f = 0.525  # cycles per unit
    t = np.arange(50000)
    u = 1e-3 * np.sin(2 * np.pi * f * t / steps_per_unit) + 1e-5 * np.sin(2 * np.pi * 3.1 * t / steps_per_unit)
    got = bench.dominant_frequency(u, L, u0)
    assert abs(got - f) < 1.0 / (len(t) / steps_per_unit)  # within one frequency bin

"""Pins of the aeroacoustic post-processing (paper_1710_02065_gb300.acoustics):
band powers against closed forms (a tone puts A^2/2 in its band; Parseval over
bands), SPL of a known amplitude, the temporal-mean removal of Delta p~, and
the 1/r extrapolation against an outgoing spherical wave."""
import math

import numpy as np

from paper_1710_02065_gb300 import acoustics as ac


def test_tone_lands_in_its_band_with_half_its_squared_amplitude():
    dt, n = 1.0 / 8192, 8192
    t = np.arange(n) * dt
    fc = ac.third_octave_centres(20.0, 4000.0)
    f0 = 1000.0  # a centre frequency and an integer number of periods in the record
    A = 0.3
    bp = ac.band_powers(A * np.sin(2 * math.pi * f0 * t) + 0.7, dt, fc)
    k = int(np.argmin(np.abs(fc - f0)))
    assert abs(bp[k] - A * A / 2) < 1e-12
    assert np.abs(np.delete(bp, k)).max() < 1e-20


def test_bands_covering_the_spectrum_add_up_to_the_variance():
    rng = np.random.default_rng(1)
    dt, n = 1e-3, 4096
    x = rng.normal(size=n)
    fc = ac.third_octave_centres(1e-3, 1e6, f_ref=1.0)
    # bands from below the first bin to above Nyquist cover every bin
    assert fc[0] * 2 ** (-1 / 6) < 1 / (n * dt) and fc[-1] * 2 ** (1 / 6) > 0.5 / dt
    assert abs(ac.band_powers(x, dt, fc).sum() - x.var()) < 1e-12 * x.var()


def test_spl_and_oaspl():
    assert abs(ac.spl(1.0, 1.0)) < 1e-15
    t = np.arange(1000) / 1000.0
    p = 2e-5 * math.sqrt(2) * np.cos(2 * math.pi * 50 * t)  # rms 20 uPa
    assert abs(ac.oaspl(p, 2e-5)) < 1e-9


def test_pressure_fluctuation_removes_the_temporal_mean():
    rng = np.random.default_rng(2)
    rho = 1.0 + 1e-3 * rng.normal(size=(64, 5)) + np.linspace(0, 1e-3, 5)
    dp = ac.pressure_fluctuation(rho)
    assert np.abs(dp.mean(axis=0)).max() < 1e-15  # round-off of rho ~ 1
    assert np.allclose(dp, (rho - rho.mean(axis=0)) / 3.0, rtol=0, atol=1e-15)


def test_far_field_follows_an_outgoing_spherical_wave():
    c, k = 1 / math.sqrt(3), 0.2
    t = np.arange(400) * 1.0
    r1, r2 = 40.0, 160.0
    wave = lambda r: np.cos(k * (r - c * t)) / r  # noqa: E731
    p2 = ac.far_field(wave(r1), r1, r2)
    # same amplitude as the wave at r2 (the phase is the retarded-time shift)
    assert abs(np.abs(p2).max() - np.abs(wave(r2)).max()) < 1e-4 / r2

"""Aeroacoustic post-processing of probe time series (host side).

The pressure signals come from the device (``lbm_probe`` per step, or the
fields of ``lbm_pressure_fluctuation``); this module turns them into the
quantities the paper reports for its cylinder and jet (Sec. III, Sec. IV):

  * the fluctuating pressure Delta p~ = Delta p - Delta p_mean of a series
    (temporal mean removed), with p = c_s^2 rho in lattice units;
  * spectra in 1/3-octave bands and the overall sound pressure level;
  * the 1/r extrapolation of a far-field signal from the probe radius to an
    observer radius (acoustic pressure of a compact source decays as 1/r).

Band powers are one-sided and normalised so that the bands covering
(0, Nyquist] add up to the variance of the signal (Parseval).
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def pressure_fluctuation(rho_series: np.ndarray, axis: int = 0) -> np.ndarray:
    """Delta p~ = c_s^2 (rho - temporal mean of rho) of a density series
    (time along `axis`)."""
    r = np.asarray(rho_series, dtype=np.float64)
    return CS2 * (r - r.mean(axis=axis, keepdims=True))


def third_octave_centres(fmin: float, fmax: float, f_ref: float = 1000.0) -> np.ndarray:
    """Base-two 1/3-octave centre frequencies f_ref 2^(k/3) in [fmin, fmax]."""
    kmin = int(np.floor(3 * np.log2(fmin / f_ref))) - 1
    kmax = int(np.ceil(3 * np.log2(fmax / f_ref))) + 1
    fc = f_ref * 2.0 ** (np.arange(kmin, kmax + 1) / 3.0)
    return fc[(fc >= fmin) & (fc <= fmax)]


def band_powers(p: np.ndarray, dt: float, centres: np.ndarray) -> np.ndarray:
    """Mean-square pressure in each 1/3-octave band [f_c 2^(-1/6), f_c 2^(1/6))
    from the one-sided periodogram of the mean-removed signal (rectangular
    window: exact for signals periodic in the record)."""
    x = np.asarray(p, dtype=np.float64)
    x = x - x.mean()
    n = len(x)
    spec = np.abs(np.fft.rfft(x)) ** 2 / n ** 2
    spec[1:] *= 2.0
    if n % 2 == 0:
        spec[-1] /= 2.0  # the Nyquist bin appears once
    f = np.fft.rfftfreq(n, dt)
    lo, hi = centres * 2.0 ** (-1.0 / 6.0), centres * 2.0 ** (1.0 / 6.0)
    return np.array([spec[(f >= a) & (f < b)].sum() for a, b in zip(lo, hi)])


def spl(power: np.ndarray | float, p_ref: float) -> np.ndarray | float:
    """Sound pressure level 10 log10(<p^2> / p_ref^2) in dB."""
    return 10.0 * np.log10(np.asarray(power) / p_ref ** 2)


def oaspl(p: np.ndarray, p_ref: float) -> float:
    """Overall sound pressure level of the mean-removed signal."""
    x = np.asarray(p, dtype=np.float64)
    return float(spl(np.mean((x - x.mean()) ** 2), p_ref))


def far_field(p: np.ndarray, r_probe: float, r_target: float) -> np.ndarray:
    """Extrapolate a far-field acoustic pressure signal from radius r_probe to
    r_target by the 1/r decay (the retarded-time shift is not applied)."""
    return np.asarray(p, dtype=np.float64) * (r_probe / r_target)

"""Pins of the charging-rate correlation of Sec. 4 (host code).

* the Re_tau of the largest rate of Eq. pysr-result, which the paper quotes as
  about 1280, 665 and 340 for 25, 50 and 100 um (this fixes d_rel in um);
* the closed-form peak equals a dense search of the correlation;
* the compact form tends to 10^-5.89 (about 1e-6, as the paper states) as
  Re_tau grows, and rises with Re_tau and with the diameter;
* at 100 um the accurate form falls beyond Re_tau = 300 (Sec. 4);
* the rate fit recovers an exact slope and ignores t+ >= 4000.
"""
import numpy as np
import pytest

from paper_2602_10761_gb300 import correlation as cor


@pytest.mark.parametrize("d_um,printed", [(25.0, 1280.0), (50.0, 665.0), (100.0, 340.0)])
def test_peak_reynolds_numbers_printed_in_sec_4(d_um, printed):
    assert abs(cor.peak_re_tau(d_um) / printed - 1) < 0.005
    re = np.linspace(100.0, 5000.0, 200_001)
    r = cor.rate(re, d_um)
    assert abs(re[np.argmax(r)] - cor.peak_re_tau(d_um)) < 0.05


def test_compact_form_asymptote_and_monotonicity():
    assert abs(cor.rate_simple(1e12, 50.0) / 10 ** -5.89 - 1) < 1e-6
    re = np.array([180.0, 300.0, 395.0, 550.0, 1000.0])
    for d in (25.0, 50.0, 100.0):
        assert np.all(np.diff(cor.rate_simple(re, d)) > 0)
    assert np.all(np.diff(cor.rate_simple(550.0, np.array([25.0, 50.0, 100.0]))) > 0)


def test_accurate_form_falls_for_large_particles_beyond_300():
    r = cor.rate(np.array([300.0, 395.0, 550.0]), 100.0)
    assert np.all(np.diff(r) < 0)
    # and still rises there for 25 um particles
    assert np.all(np.diff(cor.rate(np.array([300.0, 395.0, 550.0]), 25.0)) > 0)


def test_fit_rate_window():
    t = np.linspace(0.0, 6000.0, 61)
    q = 3e-7 * t + 1e-4
    q[t >= 4000.0] = 5.0                      # saturation beyond the window
    assert abs(cor.fit_rate(t, q) - 3e-7) <= 1e-18
    with pytest.raises(ValueError):
        cor.fit_rate([5000.0, 6000.0], [0.0, 1.0])


def test_wall_units():
    assert abs(cor.t_plus(1.0, 0.1314, 1.46e-5) - 0.1314 ** 2 / 1.46e-5) < 1e-9

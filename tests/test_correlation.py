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


class _FakeChannel:
    """Host stand-in for a Channel: the mean charge after the run is
    J = a * U_c + b * kappa_A (linear, as the condenser charge is in U_c and
    kappa_A), with the exact derivatives as the adjoint would return them."""

    def __init__(self, a=3e-17, b=-2e-17, U_c=100.0, kappa_A=1.0):
        from paper_2602_10761_gb300 import Params
        self.a, self.b = a, b
        self.params = Params(U_c=U_c, kappa_A=kappa_A)
        self.calls = 0

    def set_params(self, p):
        self.params = p

    def adjoint(self, particles, dt, nsteps, ckpt_every, want_dd=True):
        self.calls += 1
        J = self.a * self.params.U_c + self.b * self.params.kappa_A
        return J, self.a, self.b, None


@pytest.mark.parametrize("param,true", [("U_c", 2e3), ("kappa_A", 1.7)])
def test_calibrate_newton_on_a_linear_charge(param, true):
    ch = _FakeChannel()
    target = (ch.a * true + ch.b * ch.params.kappa_A if param == "U_c"
              else ch.a * ch.params.U_c + ch.b * true)
    theta, hist = cor.calibrate(ch, lambda: None, 1e-5, 10, target, param=param, iters=5, rtol=1e-12)
    # one Newton correction is exact for a linear J; the second evaluation confirms it
    assert abs(theta / true - 1) < 1e-12
    assert len(hist) == 2 and ch.calls == 2
    assert getattr(ch.params, param) == theta


def test_calibrate_rejects_a_flat_charge_and_unknown_parameters():
    ch = _FakeChannel(a=0.0)
    with pytest.raises(ArithmeticError):
        cor.calibrate(ch, lambda: None, 1e-5, 10, 1e-15, param="U_c")
    with pytest.raises(ValueError):
        cor.calibrate(_FakeChannel(), lambda: None, 1e-5, 10, 1e-15, param="rho_p")


class _FakeStepper:
    """Host stand-in for charging_history: every step adds dq to each charge."""

    def __init__(self, n, dq):
        self.n, self.dq, self.q, self.steps = n, dq, 0.0, []

    def stats(self, particles):
        return {"sum_q": self.q * self.n}

    def step(self, particles, dt, k):
        self.steps.append(k)
        self.q += self.dq * k


def test_charging_history_samples_and_rate():
    class P:
        n = 1000
    ch = _FakeStepper(P.n, dq=1e-19)
    dt, u_tau, nu = 4.2e-5, 0.1314, 1.46e-5
    tp, qrel = cor.charging_history(ch, P, dt, 25, 10, u_tau, nu)
    assert ch.steps == [10, 10, 5]                 # the last chunk is the remainder
    assert np.allclose(tp, cor.t_plus(np.array([0, 10, 20, 25]) * dt, u_tau, nu))
    assert np.allclose(qrel, np.array([0, 10, 20, 25]) * 1e-19 / cor.Q_SAT)
    # a constant rate per step gives the slope dq / (Q_SAT dt+) exactly
    slope = cor.fit_rate(tp, qrel)
    assert abs(slope / (1e-19 / cor.Q_SAT / (dt * u_tau ** 2 / nu)) - 1) < 1e-10

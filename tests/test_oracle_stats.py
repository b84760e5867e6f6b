"""Pins of the statistics reference (section 4: ionised fractions, Gamma12/J21, the
distributions (1-x)(nH) and J21(nH), photo-ionisation equilibrium under J0, J1, J4) and of the
library's host-side equilibrium curve."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from oracle import stats_oracle as S
from paper_1004_2503_b300 import aton as A

C = 2.99792458e10
SIG = 1.63e-18


def _state(shape, N, y, T, n):
    f = lambda v: np.full(shape, v, np.float32)
    return f(N), f(y), f(T), f(n)


def test_uniform_state_averages_and_single_bins():
    N, y, T, n = _state((4, 5, 6), 3e-9, 0.25, 2e4, 3e-4)
    r = S.stats(N, y, T, n, C, SIG, 1.0)
    assert r["x_volume"] == pytest.approx(0.75, rel=1e-7)
    assert r["x_mass"] == pytest.approx(0.75, rel=1e-7)
    assert r["T_volume"] == pytest.approx(2e4, rel=1e-7) and r["T_mass"] == pytest.approx(2e4, rel=1e-7)
    assert r["gamma12_volume"] == pytest.approx(C * SIG * 3e-9 / 1e-12, rel=1e-7)
    for h in (r["hist_y"], r["hist_J"]):
        assert h.sum() == 120 and (h > 0).sum() == 1
    # the occupied density bin holds n: edge[b] <= n < edge[b+1]
    E = S.edges(1e-6, 1.0, 48)
    b = int(np.nonzero(r["bin_count"])[0][0])
    assert E[b] <= np.float32(3e-4) < E[b + 1]
    assert r["bin_mean_y"][b] == pytest.approx(0.25, rel=1e-7)


def test_mass_weighting_of_a_two_phase_box():
    """Half the cells dense and neutral, half diffuse and ionised: x_v = 1/2 but the mass is
    mostly neutral, x_m = (n2 x2 + n1 x1)/(n1 + n2)."""
    shape = (2, 4, 4)
    n = np.ones(shape, np.float32) * np.float32(1e-2)
    n[1] = 1e-5
    y = np.ones(shape, np.float32)
    y[1] = 0.0
    N = np.zeros(shape, np.float32)
    T = np.full(shape, 100.0, np.float32)
    T[1] = 2e4
    r = S.stats(N, y, T, n, C, SIG, 1.0)
    n1, n2 = float(np.float32(1e-2)), float(np.float32(1e-5))
    assert r["x_volume"] == pytest.approx(0.5, rel=1e-12)
    assert r["x_mass"] == pytest.approx(n2 / (n1 + n2), rel=1e-6)
    assert r["T_mass"] == pytest.approx((n1 * 100 + n2 * 2e4) / (n1 + n2), rel=1e-6)
    assert r["J21_volume"] == 0.0
    # the ionised half sits in the lowest neutral-fraction bin (y = 0 < first edge)
    assert r["hist_y"][:, 0].sum() == 16


def test_gamma_is_the_photo_ionisation_rate_of_the_chemistry():
    """Gamma12 of a cell equals the e-folding rate of its neutral fraction under the oracle's
    chemistry when recombination is negligible and the photons are held (large reservoir)."""
    n, N, y0 = 1e-6, 1e-2, 0.9
    G = S.stats(np.float32([N]), np.float32([y0]), np.float32([1e9]), np.float32([n]),
                C, SIG, 1.0)["gamma12_volume"] * 1e-12
    t = 0.3 / G
    p = O.params(dt=t, sub_eps=1e-4, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, fixed_T=1,
                 coll_ion=0, max_sub=10 ** 7)
    r = O.chem_cell(p, n, float(np.float32(N)), [0, 0, 0], 1 - y0, 1e9)
    rate = -math.log((1 - r["x"]) / y0) / t
    assert rate == pytest.approx(G, rel=2e-3)


@pytest.mark.parametrize("alpha", [0.0, 1.0, 1.5, 3.0])
def test_J21_reading_matches_the_frequency_integral(alpha):
    """Gamma = int_{nu0}^inf 4 pi J_nu sigma_nu / (h nu) dnu for J_nu = J0 (nu/nu0)^-alpha and
    sigma = sigma0 (nu/nu0)^-3, integrated numerically, against the closed form used."""
    nu0 = 13.6 * 1.602176634e-12 / S.H_PLANCK
    J0 = 1e-21
    f = lambda u: 4 * math.pi * J0 * u ** -alpha * S.SIGMA_0 * u ** -3 / (S.H_PLANCK * u * nu0) * nu0
    val, _ = integrate.quad(f, 1.0, np.inf, epsabs=0, epsrel=1e-12)
    assert S.gamma_per_J21(alpha) == pytest.approx(val, rel=1e-9)


def test_bin_edges_decide_exactly():
    E = S.edges(1e-3, 1e3, 6)          # decades
    assert E[3] == np.float32(1.0)
    v = np.array([E[2], np.nextafter(E[2], np.float32(0)), 1e-9, 1e9, E[6], E[5]], np.float32)
    b = S.bins(v, E)
    assert list(b) == [2, 1, 0, 5, 5, 5]


def test_equilibrium_limits_and_balance():
    nH = np.geomspace(1e-7, 1.0, 61)
    T = 1e4
    for power, nstar in ((0, 1.0), (1, 0.007), (4, 0.018)):
        y = S.equilibrium_y(nH, 0.3, nstar, power, T)
        x = 1 - y
        G = 0.3 * S.gamma_per_J21(1.0) * (1 if power == 0 else np.exp(-(nH / nstar) ** power))
        # balance (1-x) G = alpha nH x^2, to rounding
        lhs, rhs = y * G, O.alpha_B(T) * nH * x * x
        assert np.allclose(lhs, rhs, rtol=1e-9)
        assert np.all(np.diff(y) >= -4 * np.finfo(float).eps)   # denser gas is more neutral
    # far below n* the self-shielded fields are the uniform one
    y0 = S.equilibrium_y(np.array([1e-8]), 0.3, 0.007, 0, T)
    y1 = S.equilibrium_y(np.array([1e-8]), 0.3, 0.007, 1, T)
    assert y1[0] == pytest.approx(y0[0], rel=1e-5)
    # at n* J1 and J4 are J0/e: the same equilibrium as a uniform field of J0/e
    for power, nstar in ((1, 0.007), (4, 0.018)):
        ys = S.equilibrium_y(np.array([nstar]), 0.3, nstar, power, T)
        yu = S.equilibrium_y(np.array([nstar]), 0.3 / math.e, 1.0, 0, T)
        assert ys[0] == pytest.approx(yu[0], rel=1e-12)
    # optically thin limit y ~ alpha nH / Gamma
    y = S.equilibrium_y(np.array([1e-6]), 10.0, 1.0, 0, T)
    assert y[0] == pytest.approx(O.alpha_B(T) * 1e-6 / (10 * S.gamma_per_J21(1.0)), rel=1e-4)
    # no field: neutral
    assert S.equilibrium_y(np.array([1e-3]), 0.0)[0] == 1.0


def test_library_equilibrium_curve_matches_the_reference():
    """Host logic of aton_equilibrium_neutral_fraction (no GPU involved)."""
    nH = np.geomspace(1e-7, 1.0, 40)
    for power, nstar, alpha in ((0, 1.0, 1.0), (1, 0.007, 1.0), (4, 0.018, 0.5)):
        ref = S.equilibrium_y(nH, 0.42, nstar, power, 2e4, alpha)
        got = A.equilibrium_neutral_fraction(nH, 0.42, nstar, power, 2e4, alpha)
        assert np.allclose(got, ref, rtol=1e-12)


def test_library_equilibrium_curve_rejects_bad_arguments():
    nH = np.array([1e-3])
    for kw in (dict(J21_0=-1.0), dict(T=0.0), dict(power=2), dict(power=4, n_star=0.0),
               dict(spectral_index=-3.0)):
        args = dict(J21_0=1.0, n_star=1.0, power=0, T=1e4, spectral_index=1.0)
        args.update(kw)
        with pytest.raises(A.AtonError):
            A.equilibrium_neutral_fraction(nH, **args)

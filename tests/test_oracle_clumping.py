"""Pins of the clumping-factor chemistry (section 3.2.1: the sub-grid clumping factors C_R
and C_I multiply the recombination and the photo-ionisation terms of the balance Eq. 14; the
clumping form Eq. 15 is read with the signs of Eq. 14). C = max(1, A nH^b) with A = 0 meaning
off; the normalisations A, b are parameters (the paper gives them only through figures)."""
import math

import pytest

import oracle as O

C = 2.99792458e10
SIG = 1.63e-18


def _p(dt, eps, **kw):
    base = dict(dt=dt, sub_eps=eps, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, fixed_T=1,
                coll_ion=0, max_sub=10 ** 6)
    base.update(kw)
    return O.params(**base)


def test_recombination_clumping_scales_the_recombination_rate():
    """Gamma = 0, T fixed: dx/dt = -C_R alpha nH x^2, x(t) = x0 / (1 + C_R alpha nH x0 t)."""
    n, x0, T, t = 2.0, 0.9, 1e4, 2e11
    A, b = 3.0, 0.7
    CR = A * n ** b
    exact = x0 / (1 + CR * O.alpha_B(T) * n * x0 * t)
    r = O.chem_cell(_p(t, 1e-3, clump_R_A=A, clump_R_b=b), n, 0.0, [0, 0, 0], x0, T)
    assert r["x"] == pytest.approx(exact, rel=2e-4)
    # the same run without clumping is far off: the factor is really applied
    r0 = O.chem_cell(_p(t, 1e-3), n, 0.0, [0, 0, 0], x0, T)
    assert abs(r0["x"] / exact - 1) > 0.1


def test_clumping_factor_is_floored_at_one():
    """A nH^b below 1 leaves the rates unclumped (the sub-grid density cannot fall below the
    mean), so the result equals the run with clumping off."""
    n, x0, T, t = 1e-3, 0.9, 1e4, 1e14
    p1 = _p(t, 1e-2, clump_R_A=2.0, clump_R_b=0.7, clump_I_A=1.5, clump_I_b=0.2)  # A n^b < 1
    p0 = _p(t, 1e-2)
    for N in (0.0, 1e-3):
        r1 = O.chem_cell(p1, n, N, [0, 0, 0], x0, T)
        r0 = O.chem_cell(p0, n, N, [0, 0, 0], x0, T)
        assert r1["x"] == r0["x"] and r1["N"] == r0["N"]


def test_ionisation_clumping_scales_the_photo_ionisation_rate():
    """No recombination: K = N - nH y is conserved and y(t) = y0 a e^{-at} / (a + b y0
    (1 - e^{-at})) with the photo-ionisation rate multiplied by C_I: a = C_I c sigma K,
    b = C_I c sigma nH."""
    n, y0, N0, t = 1.0, 0.999, 2.0, 3e3
    A, bexp = 2.5, 0.2
    CI = A * n ** bexp
    K = N0 - n * y0
    a, b = CI * C * SIG * K, CI * C * SIG * n
    e = math.exp(-a * t)
    y_exact = y0 * a * e / (a + b * y0 * (1 - e))
    # recombination switched off in effect: T so high that alpha_B is negligible over t
    r = O.chem_cell(_p(t, 1e-3, clump_I_A=A, clump_I_b=bexp), n, N0, [0, 0, 0], 1 - y0, 1e9)
    y = 1 - r["x"]
    assert y == pytest.approx(y_exact, rel=3e-3)
    # photons removed equal atoms ionised: clumping does not break the budget
    assert r["absorbed"] == pytest.approx(N0 - r["N"], rel=1e-12)
    assert (N0 - r["N"]) == pytest.approx(n * (y0 - y), rel=1e-4)


def test_clumped_equilibrium_under_a_fixed_field():
    """With photons held at N: C_I Gamma (1 - x) = C_R alpha nH x^2, so x_eq = 2G / (G +
    sqrt(G^2 + 4 a G)) with G = C_I c sigma N and a = C_R alpha nH."""
    n, T = 1e-6, 1e4
    A_R, b_R, A_I, b_I = 40.0, 0.1, 3.0, 0.05
    CR, CI = A_R * n ** b_R, A_I * n ** b_I
    assert CR > 1 and CI > 1
    N = 1e-6 * 1e4
    G = CI * C * SIG * N
    a = CR * O.alpha_B(T) * n
    x_eq = 2 * G / (G + math.sqrt(G * G + 4 * a * G))
    p = _p(1000.0 / G, 0.1, clump_R_A=A_R, clump_R_b=b_R, clump_I_A=A_I, clump_I_b=b_I)
    r = O.chem_cell(p, n, N, [0, 0, 0], 1e-3, T)
    assert r["x"] == pytest.approx(x_eq, rel=1e-6)
    # and it is not the unclumped equilibrium
    G0 = C * SIG * N
    x0 = 2 * G0 / (G0 + math.sqrt(G0 * G0 + 4 * O.alpha_B(T) * n * G0))
    assert abs((1 - x_eq) / (1 - x0) - CR / CI) < 1e-2 * CR / CI


def test_recombination_clumping_raises_recombination_cooling():
    """The clumping factor of recombinations multiplies the recombination cooling too (the
    cooling follows the recombinations it comes from); the other channels stay unclumped."""
    n, x, T = 10.0, 0.5, 2e4
    A, b = 2.0, 0.5
    CR = A * n ** b
    p1 = O.params(clump_R_A=A, clump_R_b=b, coll_ion=1)
    p0 = O.params(coll_ion=1)
    d = O.cooling_rate(p1, T, x, n) - O.cooling_rate(p0, T, x, n)
    ne = nHII = x * n
    assert d == pytest.approx((CR - 1) * O.cool_rec_B(T) * ne * nHII, rel=1e-12)

"""Pins of the oracle's chemistry/cooling/absorption operator (Appendix Eq. A4; section 2.2
chemistry paragraph; ionisation balance of section 3.2.1, Eq. 14) and of its rate fits."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KB = 1.380649e-16
EV = 1.602176634e-12
C = 2.99792458e10
SIG = 1.63e-18


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ----------------------------------------------------------------------------------- rates
def test_alpha_B_matches_textbook_table():
    for T, a in _table("osterbrock_alpha_B.txt"):
        assert O.alpha_B(float(T)) == pytest.approx(float(a), rel=0.02)


def test_collisional_ionisation_matches_independent_fit():
    v = {r[0]: float(r[1]) for r in _table("voronov1997_H.txt")}
    kev = 8.617333262e-5
    for T, tol in ((2e4, 0.2), (5e4, 0.1), (1e5, 0.06), (3e5, 0.06), (1e6, 0.06)):
        U = v["dE_eV"] / (kev * T)
        ref = v["A"] * (1 + v["P"] * math.sqrt(U)) * U ** v["K"] * math.exp(-U) / (v["X"] + U)
        assert O.beta_coll(T) == pytest.approx(ref, rel=tol), T


def test_collisional_excitation_cooling_matches_collision_strengths():
    """Cen (1992) H I collisional-excitation cooling against the energy lost through the
    1s -> 2s and 1s -> 2p excitations computed from tabulated effective collision strengths,
    E12 q12 with q12 = 8.629e-6 Upsilon exp(-E12/kT) / (g1 sqrt(T)). The fit also holds the
    (smaller) excitations to n >= 3, so it lies at or a little above the n = 2 sum: the ratio
    stays within [0.8, 1.3] from 5000 K to 20000 K. Over that range the Boltzmann factor alone
    changes by eight decades, so a wrong threshold temperature, prefactor or temperature
    divisor leaves the window."""
    kev = 8.617333262e-5
    e12 = 10.20                      # eV
    ratios = []
    for T, u2s, u2p in _table("hi_collision_strengths.txt"):
        T = float(T)
        q12 = 8.629e-6 / (2.0 * math.sqrt(T)) * (float(u2s) + float(u2p)) * math.exp(-e12 / (kev * T))
        ratios.append(O.cool_coll_exc(T) / (e12 * EV * q12))
    assert all(0.8 <= r <= 1.3 for r in ratios), ratios
    # the n >= 3 share grows with temperature: the ratio does not fall from 5000 K to 20000 K
    assert ratios[-1] >= ratios[0]


def test_bremsstrahlung_gaunt_factor_in_textbook_range():
    # free-free emissivity 1.42e-27 g sqrt(T) n_e n_p with a Gaunt factor of order 1.1-1.5
    for T in (1e4, 1e5, 1e6, 1e7):
        g = O.cool_brems(T) / (1.42e-27 * math.sqrt(T))
        assert 1.1 <= g <= 1.45


def test_recombination_cooling_energy_per_recombination():
    # mean kinetic energy carried away per recombination is a fraction of kT (slow electrons
    # recombine preferentially): between 0.4 and 0.9 kT from 1e3 to 1e5 K
    for T in (1e3, 1e4, 1e5):
        r = O.cool_rec_B(T) / (O.alpha_B(T) * KB * T)
        assert 0.4 < r < 0.9
    # and the fraction falls with temperature
    assert (O.cool_rec_B(1e3) / (O.alpha_B(1e3) * 1e3) > O.cool_rec_B(1e4) / (O.alpha_B(1e4) * 1e4)
            > O.cool_rec_B(1e5) / (O.alpha_B(1e5) * 1e5))


def _kramers_milne_case_B(T, nmax=2000):
    """Case-B recombination rate alpha_B [cm^3 s^-1] and kinetic-energy loss coefficient
    beta_B [cm^3 s^-1, times kT] of hydrogen from first principles: Kramers' bound-free cross
    section of level n (all l), sigma_n(nu) = 7.907e-18 n (nu_n/nu)^3 cm^2 (Gaunt factor 1),
    turned into a recombination cross section by the Milne relation with g_n = 2 n^2, g_+ = 1,
    sigma_rec = g_n (h nu / m_e c v)^2 sigma_n, and averaged over a Maxwellian. With
    E = m_e v^2 / 2 and h nu = chi_n + E the Maxwellian integrals close in the exponential
    integral: with x_n = chi_n / kT and s_n = exp(x_n) E1(x_n),
      alpha_n = K n^3 chi_n^3 (kT)^-3/2 s_n,  beta_n = K n^3 chi_n^3 (kT)^-3/2 (1 - x_n s_n),
    K = 2 sigma_0 sqrt(2/m_e) / (sqrt(pi) m_e c^2); case B sums n >= 2."""
    from scipy.special import exp1
    me, ry = 9.1093837e-28, 13.605693 * EV
    kT = KB * T
    n = np.arange(2, nmax + 1, dtype=np.float64)
    chi = ry / n ** 2
    x = chi / kT
    s = np.exp(x) * exp1(x)
    K = 2.0 * 7.907e-18 * math.sqrt(2.0 / me) / (math.sqrt(math.pi) * me * C ** 2)
    pre = K * n ** 3 * chi ** 3 * kT ** -1.5
    return float(np.sum(pre * s)), float(np.sum(pre * (1.0 - x * s)))


def test_recombination_cooling_against_kramers_milne():
    """The Hui & Gnedin (1997) case-B recombination-cooling fit against an independent
    first-principles calculation (Kramers cross sections, Milne relation, Maxwellian; see
    _kramers_milne_case_B). The mean kinetic energy carried off per recombination,
    Lambda_B / (alpha_B kT), does not depend on the cross sections' normalisation and agrees
    within 3 % from 3000 to 30 000 K (0.66 kT at 1e4 K); the energy-loss coefficient itself,
    Lambda_B / kT, agrees with beta_B within 8 % (Gaunt factors near one for the excited
    levels). A wrong exponent or divisor of the fit moves it far outside either window."""
    for T in (3e3, 5e3, 1e4, 2e4, 3e4):
        a_km, b_km = _kramers_milne_case_B(T)
        lam = O.cool_rec_B(T)
        assert lam / (O.alpha_B(T) * KB * T) == pytest.approx(b_km / a_km, rel=0.03), T
        assert lam / (KB * T) == pytest.approx(b_km, rel=0.08), T
    # the reference itself: Kramers' alpha_B is within 5 % of the textbook case-B values
    for T, a in _table("osterbrock_alpha_B.txt"):
        if 5e3 <= float(T) <= 2e4:
            assert _kramers_milne_case_B(float(T))[0] == pytest.approx(float(a), rel=0.05)


def test_heat_per_ionisation_from_paper_constants():
    g = {r[0]: float(r[1]) for r in _table("paper_constants.txt")}
    p = O.params(sigma_n=g["sigma_n"], sigma_e=g["sigma_e"], e_gamma_eV=g["e_gamma"])
    assert O.heat_per_ionisation(p) / EV == pytest.approx(g["heat_per_ionisation"], rel=1e-9)
    # workloads: sigma_e = sigma_n, 29.6 eV photons leave 16.0 eV per ionisation
    p2 = O.params(sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6)
    assert O.heat_per_ionisation(p2) / EV == pytest.approx(16.0, rel=1e-12)


# ------------------------------------------------------------------------- closed forms
def _chem(dt, eps, **kw):
    base = dict(dt=dt, sub_eps=eps, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, fixed_T=1,
                coll_ion=0, max_sub=10 ** 6)
    base.update(kw)
    return O.params(**base)


def test_recombination_only_closed_form_and_first_order_convergence():
    """Gamma = 0, T fixed: dx/dt = -alpha nH x^2, so x(t) = x0 / (1 + alpha nH x0 t)."""
    n, x0, T, t = 1.0, 0.9, 1e4, 1e12
    a = O.alpha_B(T)
    exact = x0 / (1 + a * n * x0 * t)
    errs = []
    for eps in (1e-2, 1e-3):
        r = O.chem_cell(_chem(t, eps), n, 0.0, [0, 0, 0], x0, T)
        errs.append(abs(r["x"] - exact) / exact)
        assert r["N"] == 0.0 and r["absorbed"] == 0.0
    assert errs[1] < 2e-4
    assert 5 < errs[0] / errs[1] < 20      # first-order backward differences


def test_photoionisation_without_recombination_closed_form():
    """N and y obey dN/dt = nH dy/dt = -c sigma nH y N; K = N - nH y is conserved and
    y(t) = y0 a e^{-at} / (a + b y0 (1 - e^{-at})), a = c sigma K, b = c sigma nH."""
    n, y0, N0, t = 1e-3, 0.999, 2e-3, 1e10
    K = N0 - n * y0
    a, b = C * SIG * K, C * SIG * n
    e = math.exp(-a * t)
    y_exact = y0 * a * e / (a + b * y0 * (1 - e))
    r = O.chem_cell(_chem(t, 1e-3), n, N0, [0, 0, 0], 1 - y0, 1e4)
    y = 1 - r["x"]
    assert y == pytest.approx(y_exact, rel=2e-3)
    # photons removed equal atoms ionised, up to the (tiny) recombinations
    assert r["absorbed"] == pytest.approx(N0 - r["N"], rel=1e-12)
    assert (N0 - r["N"]) == pytest.approx(n * (y0 - y), rel=1e-4)


def test_flux_decays_with_the_photon_density():
    r = O.chem_cell(_chem(1e10, 0.1), 1e-3, 2e-3, [3e7, -1e7, 2e7], 0.001, 1e4)
    assert np.allclose(r["F"] / np.array([3e7, -1e7, 2e7]), r["N"] / 2e-3, rtol=1e-12)


def test_photoionisation_equilibrium_uniform_injection():
    """Periodic uniform box, one identical source in every cell, T fixed, no collisions: at
    steady state the recombinations balance the emission, alpha nH^2 x^2 = Ndot / V."""
    n, T = 1.0, 1e4
    a = O.alpha_B(T)
    x_eq = 0.5
    Ndot_over_V = a * n * n * x_eq ** 2
    dt = 0.01 / (a * n)
    p = _chem(dt, 0.1, dx=1.0, bc=O.BC_PERIODIC)
    shape = (3, 3, 3)
    st = dict(N=np.zeros(shape), Fx=np.zeros(shape), Fy=np.zeros(shape), Fz=np.zeros(shape),
              x=np.full(shape, 1e-3), T=np.full(shape, T), nH=np.full(shape, n))
    idx = np.arange(27)
    out, b, s = O.run(p, st, 3000, idx, np.full(27, Ndot_over_V))
    assert out["x"] == pytest.approx(np.full(shape, x_eq), rel=2e-3)


def test_equilibrium_formula_under_a_fixed_field():
    """With photons held (re-supplied) at N, x_eq solves Gamma (1 - x) = alpha nH x^2:
    y_eq = alpha nH x_eq^2 / Gamma with x_eq = 2 Gamma / (Gamma + sqrt(Gamma^2 + 4 alpha nH
    Gamma)). Emulated with a very large photon reservoir relative to the atoms."""
    n, T = 1e-6, 1e4
    a = O.alpha_B(T)
    N = 1e-6 * 1e4       # 1e4 photons per atom: absorption changes N by < 1e-4
    G = C * SIG * N
    x_eq = 2 * G / (G + math.sqrt(G * G + 4 * a * n * G))
    r = O.chem_cell(_chem(1000.0 / G, 0.1), n, N, [0, 0, 0], 1e-3, T)
    assert r["x"] == pytest.approx(x_eq, rel=1e-9)
    G1 = C * SIG * r["N"]          # the reservoir lost 1e-4 of its photons
    y_eq = a * n * r["x"] ** 2 / G1
    assert 1 - r["x"] == pytest.approx(y_eq, rel=1e-3)


def test_energy_conservation_with_cooling_off():
    """Without cooling the thermal energy 1.5 nH (1+x) kB T grows by the photo-heating of
    the absorbed photons only."""
    p = O.params(dt=3e11, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, cooling=0, coll_ion=0)
    n, x0, T0, N0 = 1e-3, 1e-3, 100.0, 5e-4
    r = O.chem_cell(p, n, N0, [0, 0, 0], x0, T0)
    e0 = 1.5 * n * (1 + x0) * KB * T0
    e1 = 1.5 * n * (1 + r["x"]) * KB * r["T"]
    assert e1 - e0 == pytest.approx(r["absorbed"] * O.heat_per_ionisation(p), rel=1e-12)
    assert r["nsub"] > 5   # photo-heating from 100 K forces sub-cycling


def test_cooling_is_monotone_without_radiation():
    p = O.params(dt=1e13, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6)
    n, x, T, N = 1.0, 1 - 1e-6, 1e6, 0.0
    prev = T
    for _ in range(40):
        r = O.chem_cell(p, n, N, [0, 0, 0], x, prev)
        assert r["T"] <= prev and r["T"] >= p.T_floor
        x, prev = r["x"], r["T"]
    assert prev < 0.5e6


def test_subcycle_cap_sets_the_error_flag():
    p = O.params(dt=3e11, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, max_sub=3)
    r = O.chem_cell(p, 1e-3, 5e-4, [0, 0, 0], 1e-3, 100.0)
    assert r["err"] == 1 and r["nsub"] == 3


def test_result_is_continuous_in_the_step_length():
    """The sub-step rule (largest h up to the remaining time) makes the update continuous in
    dt even where the number of sub-steps changes."""
    n, N0, x0, T0 = 1e-3, 3e-4, 1e-3, 100.0
    dts = np.linspace(5.8e10, 6.6e10, 401)
    xs, Ts, ns = [], [], []
    for dt in dts:
        r = O.chem_cell(O.params(dt=dt, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6), n, N0,
                        [0, 0, 0], x0, T0)
        xs.append(r["x"]); Ts.append(r["T"]); ns.append(r["nsub"])
    xs, Ts = np.array(xs), np.array(Ts)
    assert len(set(ns)) > 1            # the window crosses a change of sub-step count
    assert np.abs(np.diff(xs)).max() < 1e-3
    assert np.abs(np.diff(Ts) / Ts[1:]).max() < 1e-3


def test_gas_at_the_floor_that_would_cool_takes_one_substep():
    """T cannot fall below the floor, so the temperature condition of the sub-step rule does
    not apply there: a cold cell with nothing to heat it finishes in one sub-step."""
    p = O.params(dt=1e11, sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6)
    r = O.chem_cell(p, 1e-3, 0.0, [0, 0, 0], 1e-4, p.T_floor)
    assert r["err"] == 0 and r["nsub"] == 1
    assert r["T"] == pytest.approx(p.T_floor, rel=1e-6)


def test_one_quiet_substep_is_the_quadratic_the_kernels_solve_in_closed_form():
    """With recombinations and collisional terms negligible (hot, fixed T; a = b = 0), one
    implicit sub-step y' - y = -c sigma N' y' h with N' = N / (1 + m y') is the quadratic
    m y'^2 + (1 + kN - m y) y' - y = 0 (m = nH c sigma h, kN = c sigma N h). The oracle's
    Newton step must land on its root, taken here in the cancellation-free form for either sign
    of B = 1 + kN - m y, with d = kN y' / (1 + m y') (the form the fused kernels evaluate)."""
    T = 1e6
    cases = [(1e-8, 1e10, 0.01), (1e-8, 1e10, 0.5), (1.0, 1e8, 0.05), (1.0, 1e8, 0.5),
             (3e-3, 1e10, 0.2)]
    for n, dt, kN in cases:
        y = 0.9
        N = kN / (C * SIG * dt)
        m = n * C * SIG * dt
        B = 1 + kN - m * y
        sD = math.sqrt(B * B + 4 * m * y)
        Yq = 2 * y / (B + sD) if B >= 0 else (sD - B) / (2 * m)
        d = kN * Yq / (1 + m * Yq)
        y_cf = y - d
        r = O.chem_cell(_chem(dt, 1.0), n, N, [0, 0, 0], 1 - y, T)
        assert r["nsub"] == 1, (n, dt, kN)
        # the recombinations left out of the quadratic, alpha nH dt x'^2, bound the difference
        tol = 2 * O.alpha_B(T) * n * dt * (1 - y_cf) ** 2 + 1e-12
        assert abs((1 - r["x"]) - y_cf) <= tol, (n, dt, kN, 1 - r["x"], y_cf)
        assert r["N"] == pytest.approx(N / (1 + m * y_cf), rel=1e-9 + 10 * tol)
        assert (B < 0) == (m * y > 1 + kN)
    # both signs of B are covered
    assert any(n * C * SIG * dt * 0.9 > 1 + kN for n, dt, kN in cases)

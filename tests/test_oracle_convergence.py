"""Convergence pins of the oracle's sub-cycled chemistry operator (Appendix Eq. A4; section
2.2, chemistry paragraph; the balance of section 3.2.1, Eq. 14).

The paper fixes the continuous equations the sub-cycling integrates but no sub-step rule. The
oracle's rule (each sub-step bounded by the ionisation time and by the heating and the cooling
times, eps = sub_eps) is a reading; these tests show that it does not change what the operator
converges to. As eps -> 0 the oracle must approach, at first order (backward differences):

* the solution of the same ordinary differential equations computed by an independent
  integrator (scipy's Radau at rtol 1e-11), with the oracle's own rate coefficients, for a
  photo-heated cell with cooling and collisional ionisation on;
* the closed-form Riccati solution x(t) of dx/dt = Gamma (1 - x) - alpha nH x^2 under a
  constant field (T fixed), at several times along the approach to equilibrium.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O

C = 2.99792458e10
SIG = 1.63e-18
KB = 1.380649e-16


def _params(**kw):
    base = dict(sigma_n=SIG, sigma_e=SIG, e_gamma_eV=29.6, max_sub=10 ** 8)
    base.update(kw)
    return O.params(**base)


def _ode_reference(p, n, N0, x0, T0, times):
    """(N, x, T) at ``times`` of the continuous system the operator discretises:
    dN/dt = -nH c sigma N y, dy/dt = -c sigma N y + alpha nH x^2 - beta nH x y,
    dE/dt = nH c sigma N y e_heat - Lambda(T, x, nH), E = 1.5 nH (1 + x) kB T."""
    eh = O.heat_per_ionisation(p)

    def rhs(_t, s):
        N, y, E = s
        y = min(max(y, 0.0), 1.0)
        x = 1.0 - y
        T = E / (1.5 * n * (1.0 + x) * KB)
        G = C * SIG * N
        a = O.alpha_B(T)
        b = O.beta_coll(T) if p.coll_ion else 0.0
        return [-n * G * y, -G * y + a * n * x * x - b * n * x * y,
                n * G * y * eh - O.cooling_rate(p, T, x, n)]

    E0 = 1.5 * n * (1.0 + x0) * KB * T0
    sol = solve_ivp(rhs, (0.0, times[-1]), [N0, 1.0 - x0, E0], method="Radau", rtol=1e-11,
                    atol=[N0 * 1e-14, 1e-16, E0 * 1e-14], t_eval=times)
    assert sol.success
    out = []
    for i in range(len(times)):
        N, y, E = sol.y[:, i]
        x = 1.0 - y
        out.append((N, x, E / (1.5 * n * (1.0 + x) * KB)))
    return out


def test_photo_heated_cell_with_cooling_converges_to_the_ode_at_first_order():
    """Cold, nearly neutral gas (100 K, x = 1e-4) under two photons per atom: it is
    photo-ionised and heated to ~6e4 K, where collisional ionisation and cooling act. At three
    times along the way the errors in x, T and N against the ODE halve with eps."""
    n, N0, x0, T0 = 1e-3, 2e-3, 1e-4, 100.0
    times = [2e10, 1e11, 5e11]
    ref = _ode_reference(_params(), n, N0, x0, T0, times)
    epss = (0.1, 0.05, 0.025, 0.0125)
    err = np.zeros((len(epss), len(times), 3))
    for ie, eps in enumerate(epss):
        for it, (t, (N, x, T)) in enumerate(zip(times, ref)):
            r = O.chem_cell(_params(dt=t, sub_eps=eps), n, N0, [0, 0, 0], x0, T0)
            assert r["err"] == 0
            err[ie, it] = (abs(r["x"] - x), abs(r["T"] / T - 1), abs(r["N"] / N - 1))
    ratio = err[:-1] / err[1:]
    # first order in eps; x at the last time (y ~ 1e-6, absolute error ~1e-9) is where the
    # sub-step's floor y_floor = 1e-6 on the ionisation time takes over from eps y: it still
    # falls by more than 1.4 per halving
    first = np.ones(ratio.shape, bool)
    first[:, -1, 0] = False
    assert np.all((ratio[first] > 1.7) & (ratio[first] < 2.3)), ratio
    assert np.all(ratio[:, -1, 0] > 1.4), ratio
    assert err[-1, :, 0].max() < 2e-3                             # x
    assert err[-1, :, 1].max() < 2e-3                             # T
    assert err[-1, :, 2].max() < 2e-3                             # N
    # the default eps = 0.1 is already within 1.3e-2 in x and 1e-2 in T and N
    assert err[0, :, 0].max() < 1.3e-2 and err[0, :, 1:].max() < 1.1e-2


def _riccati_y(t, G, A, x0):
    """y = 1 - x of dx/dt = G (1 - x) - A x^2: with the roots x+ > 0 > x- of A x^2 + G x - G,
    (x - x+)/(x - x-) decays as exp(-A (x+ - x-) t). Written without cancellation in y."""
    D = math.sqrt(G * G + 4 * A * G)
    xp = 2 * G / (G + D)
    xm = -(G + D) / (2 * A)
    yp = A * xp * xp / G                   # 1 - x+ from the balance G (1 - x+) = A x+^2
    e = (x0 - xp) / (x0 - xm) * math.exp(-D * t)
    return (yp - (1 - xm) * e) / (1 - e), yp


def test_fixed_field_riccati_closed_form_at_several_times():
    """T fixed, no collisional ionisation, a field with five photons per atom in nearly
    ionised gas: the photons removed over the run are < 5e-6 of N, so Gamma is constant to
    that level and y(t) follows the Riccati solution from y0 = 1e-5 towards y_eq = 1e-6.
    The relative error in y halves with eps (first order) during the approach and is below
    1.5e-3 at eps = 1/640 at every time, equilibrium included."""
    n, T = 1e-3, 1e4
    A = O.alpha_B(T) * n
    G = A / 1e-6
    N = G / (C * SIG)
    x0 = 1.0 - 1e-5
    times = [0.3 / G, 1.0 / G, 3.0 / G, 10.0 / G]
    epss = (0.1, 0.025, 0.00625, 0.0015625)
    rel = np.zeros((len(epss), len(times)))
    for ie, eps in enumerate(epss):
        for it, t in enumerate(times):
            p = _params(dt=t, sub_eps=eps, fixed_T=1, coll_ion=0, y_floor=1e-12)
            r = O.chem_cell(p, n, N, [0, 0, 0], x0, T)
            assert r["err"] == 0 and 1 - r["N"] / N < 5e-6
            ye, _ = _riccati_y(t, G, A, x0)
            rel[ie, it] = abs((1 - r["x"]) / ye - 1)
    ratio = rel[:-1, :3] / rel[1:, :3]      # eps / 4 each time: first order gives ~4
    assert np.all((ratio > 3.3) & (ratio < 4.7)), ratio
    assert np.all(rel[1:, 3] < rel[:-1, 3])  # at equilibrium: monotone convergence
    assert rel[-1].max() < 1.5e-3
    # the last time lies on the equilibrium of the fixed field (to 1e-3)
    ye, yp = _riccati_y(times[-1], G, A, x0)
    assert ye == pytest.approx(yp, rel=1e-3)

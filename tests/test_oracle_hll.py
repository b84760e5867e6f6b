"""Pins of the oracle's HLL intercell flux (section 2.2 names HLL beside Lax-Friedrichs): the
closed-form wave speeds against the eigenvalues of a finite-difference Jacobian of the oracle's
own flux, and properties of the exact solution the HLL scheme keeps (a collimated beam does
not spread sideways; uniform states stay put; photons are conserved)."""
import numpy as np
import pytest

import oracle as O

C = 2.99792458e10


def _flux(u, d, c):
    """Physical flux along d of u = (N, Fx, Fy, Fz): (F_d, c^2 N D[:, d])."""
    D = O.eddington(u[0], u[1:], c)
    return np.concatenate([[u[1 + d]], c * c * u[0] * D[:, d]])


def _jacobian(u, d, c, h=1e-7):
    J = np.zeros((4, 4))
    scale = np.array([u[0], c * u[0], c * u[0], c * u[0]])
    for k in range(4):
        e = np.zeros(4)
        e[k] = h * scale[k]
        J[:, k] = (_flux(u + e, d, c) - _flux(u - e, d, c)) / (2 * e[k])
    return J


def test_wave_speeds_are_the_extreme_jacobian_eigenvalues():
    rng = np.random.default_rng(0)
    c = 1.0
    worst = 0.0
    for _ in range(300):
        f = rng.uniform(0.02, 0.97)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u = np.concatenate([[1.0], c * f * n])
        for d in range(3):
            ev = np.linalg.eigvals(_jacobian(u, d, c)).real
            lo, hi = O.m1_speeds(u[0], u[1:], c, d)
            worst = max(worst, abs(lo - ev.min()), abs(hi - ev.max()))
    assert worst < 1e-6, worst


def test_wave_speed_limits():
    lo, hi = O.m1_speeds(2.0, [0, 0, 0], C, 1)
    assert lo == pytest.approx(-C / np.sqrt(3)) and hi == pytest.approx(C / np.sqrt(3))
    # free streaming along x: every wave moves with the photons
    lo, hi = O.m1_speeds(1.0, [C, 0, 0], C, 0)
    assert lo == pytest.approx(C) and hi == pytest.approx(C)
    lo, hi = O.m1_speeds(1.0, [C, 0, 0], C, 2)
    assert abs(lo) < 1e-6 * C and abs(hi) < 1e-6 * C
    # the speeds flip with the flux
    a = O.m1_speeds(1.0, [0.3 * C, 0.2 * C, 0], C, 0)
    b = O.m1_speeds(1.0, [-0.3 * C, -0.2 * C, 0], C, 0)
    assert a[0] == pytest.approx(-b[1]) and a[1] == pytest.approx(-b[0])


def _p(flux, dx=1.0, dt=0.3):
    return O.params(c=1.0, dx=dx, dt=dt, flux=flux)


def test_free_streaming_field_has_no_transverse_transport_under_hll():
    """Where every cell streams along x at f = 1 (a bright beam in a faint field streaming the
    same way), the exact solution only translates along x. HLL's transverse speeds are then zero
    and nothing crosses the y or z faces; the Lax-Friedrichs flux diffuses the beam sideways at
    speed c. Along x HLL is upwinding: the beam's mean position advances at c."""
    shape = (5, 9, 24)
    N = np.full(shape, 1e-3)
    N[2, 4, 2:6] = 1.0
    F = [N.copy(), np.zeros(shape), np.zeros(shape)]      # Fx = c N, c = 1
    out_h = O.transport(_p(O.FLUX_HLL), N, *F)
    out_g = O.transport(_p(O.FLUX_GLF), N, *F)
    side = (slice(None), [3, 5], slice(None))
    assert np.array_equal(out_h[0][side], N[side])
    assert np.abs(out_g[0][side] - N[side]).max() > 1e-2
    for k in (2, 3):
        assert np.abs(out_h[k]).max() == 0.0
    xs = np.arange(shape[2])
    beam = np.zeros(shape, bool)
    beam[2, 4, :] = True
    w0, w1 = (N - 1e-3)[beam], (out_h[0] - 1e-3)[beam]
    assert (xs * w1).sum() / w1.sum() - (xs * w0).sum() / w0.sum() == pytest.approx(0.3, rel=1e-9)


def test_hll_transport_conserves_photons_and_uniform_states():
    rng = np.random.default_rng(1)
    shape = (6, 7, 8)
    N = rng.uniform(0.5, 1.5, shape)
    g = rng.normal(size=(3,) + shape)
    g *= rng.uniform(0, 0.95, shape) / np.linalg.norm(g, axis=0)
    F = [g[k] * N for k in range(3)]
    out = O.transport(_p(O.FLUX_HLL), N, *F)
    assert out[0].sum() == pytest.approx(N.sum(), rel=1e-13)
    for k in range(3):
        assert out[1 + k].sum() == pytest.approx(F[k].sum(), rel=1e-12, abs=1e-12)
    Nu = np.full(shape, 0.7)
    Fu = [np.full(shape, 0.2), np.full(shape, -0.3), np.full(shape, 0.1)]
    out = O.transport(_p(O.FLUX_HLL), Nu, *Fu)
    assert np.allclose(out[0], Nu, rtol=1e-14) and np.allclose(out[2], Fu[1], rtol=1e-14)

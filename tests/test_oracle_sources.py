"""Pins of the post-processing source model (section 2.3: lifetime dilution over snapshot
intervals, nearest grid point, escape fraction and boost factor, Eqs. 16-17) and the library's
host implementation of it (no GPU involved)."""
import math

import numpy as np
import pytest

from oracle import sources_oracle as S
from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import workloads as W

MYR = W.MYR


def _star(age, L, mass=1e38, q=5e4, x=0.0, y=0.0, z=0.0):
    return dict(x=x, y=y, z=z, mass=mass, age=age, lifetime=L, photons_per_baryon=q)


@pytest.mark.parametrize("birth_frac,L_over_D", [(0.3, 7.4), (0.0, 3.0), (0.99, 0.4),
                                                 (0.5, 1.0), (0.25, 12.25)])
def test_every_star_emits_its_photons_exactly_once(birth_frac, L_over_D):
    """Over the successive snapshot intervals of its life a star's emission, rate x interval
    summed, is its total yield q M / m_H: the dilution neither loses nor duplicates photons,
    whether it is born, or dies, inside an interval, or lives less than one."""
    D = 2.0 * MYR
    L = L_over_D * D
    t_birth = birth_frac * D          # inside interval 0 = [0, D]
    star = _star(0.0, L)
    total = 0.0
    for p in range(int(L_over_D) + 3):
        star["age"] = (p + 1) * D - t_birth          # age at the end of interval p
        total += S.star_rate(star, D) * D
    Q = star["photons_per_baryon"] * star["mass"] / S.M_H
    assert total == pytest.approx(Q, rel=1e-12)


def test_dilution_cases():
    D, L = 4.0, 10.0
    nd = 1.0
    mk = lambda age: dict(mass=S.M_H * L, age=age, lifetime=L, photons_per_baryon=1.0)   # Ndot = 1
    # born a quarter of the interval before its end: emits for 1 of 4
    assert S.star_rate(mk(1.0), D) == pytest.approx(0.25 * nd)
    # active over the whole interval
    assert S.star_rate(mk(6.0), D) == pytest.approx(nd)
    # dies half-way through the interval (age L - 2 at its start)
    assert S.star_rate(mk(L - 2.0 + D), D) == pytest.approx(0.5 * nd)
    # already dead at the start
    assert S.star_rate(mk(L + D), D) == 0.0 and S.star_rate(mk(L + D + 1), D) == 0.0


def test_boost_factor_of_the_parameter_table():
    """The boost compensates unresolved star formation (SFR_converged / SFR_actual >= 1): with
    the table's a_b, k_b it is large early and tends to max(1, a_b) late; it never lowers a
    luminosity."""
    for a_b, k_b in ((0.7, 300.0), (1.0, 650.0), (1.2, 1500.0), (1.2, 3000.0)):
        ts = np.geomspace(150.0, 13000.0, 200)          # Myr
        B = np.array([S.boost(t, a_b, k_b) for t in ts])
        assert np.all(B >= 1.0)
        assert np.all(np.diff(B) <= 0)                  # falls as the Universe ages
        assert B[-1] == pytest.approx(max(1.0, a_b * math.exp(k_b / 13000.0)), rel=1e-12)
    assert S.boost(500.0, 1.2, 3000.0) == pytest.approx(1.2 * math.exp(6.0))
    assert S.boost(1.0, 0.0, 5.0) == 1.0


def test_nearest_grid_point_with_periodic_wrap():
    shape, dx = (4, 5, 6), 2.0
    assert S.star_cell(_star(1, 1, x=0.5, y=0.5, z=0.5), shape, dx) == 0
    assert S.star_cell(_star(1, 1, x=11.9, y=9.99, z=7.9), shape, dx) == 5 + 6 * (4 + 5 * 3)
    assert S.star_cell(_star(1, 1, x=-0.1, y=10.0, z=8.0), shape, dx) == 5 + 6 * (0 + 5 * 0)


def test_library_matches_the_reference_on_a_snapshot_sequence():
    st, snaps, run, interval, model = W.snapshot_workload(n_snap=4)
    shape = st["nH"].shape
    for p in range(1, len(snaps)):
        stars = snaps[p]
        t = model["t0"] + (p - 0.5) * interval
        cell, rate = A.star_sources(stars, shape, run["dx"], interval, model["f_esc"],
                                    model["boost_a"], model["boost_k"], t)
        rc, rr = S.star_sources(stars, shape, run["dx"], interval, f_esc=model["f_esc"],
                                a_b=model["boost_a"], k_b=model["boost_k"], t_universe=t)
        assert list(cell) == rc
        assert np.allclose(rate, rr, rtol=1e-14, atol=0)
    # and on stars covering every case, with lifetimes shorter than the interval
    rng = np.random.default_rng(3)
    n = 500
    stars = np.zeros(n, A.STAR_DTYPE)
    stars["x"], stars["y"], stars["z"] = (rng.uniform(-3e22, 3e22, n) for _ in range(3))
    stars["mass"] = rng.uniform(0, 1e38, n)
    stars["age"] = rng.uniform(0, 30 * MYR, n)
    stars["lifetime"] = rng.uniform(0.5, 20, n) * MYR
    stars["photons_per_baryon"] = rng.uniform(24000, 98000, n)
    for D in (0.3 * MYR, 5 * MYR):
        cell, rate = A.star_sources(stars, (8, 9, 10), 1e21, D, 0.2, 1.2, 3000 * MYR, 700 * MYR)
        rc, rr = S.star_sources(stars, (8, 9, 10), 1e21, D, f_esc=0.2, a_b=1.2,
                                k_b=3000 * MYR, t_universe=700 * MYR)
        assert list(cell) == rc
        assert np.allclose(rate, rr, rtol=1e-14, atol=0)
        assert (cell < 0).any() and (cell >= 0).any()


def test_library_rejects_bad_source_inputs():
    good = np.zeros(1, A.STAR_DTYPE)
    good["mass"], good["age"], good["lifetime"], good["photons_per_baryon"] = 1e38, 1.0, 2.0, 1e4
    A.star_sources(good, (2, 2, 2), 1.0, 1.0)
    for field, val in (("lifetime", 0.0), ("age", -1.0), ("mass", np.nan), ("x", np.inf),
                       ("photons_per_baryon", -2.0)):
        bad = good.copy()
        bad[field] = val
        with pytest.raises(A.AtonError):
            A.star_sources(bad, (2, 2, 2), 1.0, 1.0)
    for kw in (dict(interval=0.0), dict(f_esc=-0.1), dict(t_universe=0.0)):
        args = dict(interval=1.0, f_esc=1.0, t_universe=1.0)
        args.update(kw)
        with pytest.raises(A.AtonError):
            A.star_sources(good, (2, 2, 2), 1.0, **args)

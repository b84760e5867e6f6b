"""FP64 reference of the post-processing source model -- TEST INFRASTRUCTURE ONLY.

Section 2.3: the star particles of snapshot p+1 emit over [t_p, t_{p+1}] (length D); each star's
photons emitted inside the interval are spread over the whole interval. A star of mass M,
lifetime L and yield q photons per stellar baryon emits Q = q M / m_H photons uniformly over its
lifetime, Ndot = Q / L. With a its age at t_{p+1} and a_p = a - D its age at t_p:
  - a_p >= L: discarded (no emission);
  - a_p < 0: created inside the interval; it emits from its birth to t_{p+1}, or to its death if
    sooner: for min(a, L);
  - 0 <= a_p < L: it emits from t_p to t_{p+1}, or to its death at age L if sooner: for
    min(D, L - a_p);
and its rate is (emitting time / D) Ndot. Readings: the printed "(a_{p+1} - a*)" and
"min(1, L - a_p)" are read as the emitting time inside the interval (the printed forms mix
ages, times and pure numbers). The effective rate is rate * f_esc * B(t) (Eq. 16), with the
boost B(t) = max(1, a_b exp(k_b / t)) (Eq. 17 prints min, under which nothing is ever boosted),
t the age of the Universe. Stars go to their nearest grid point: cell floor(x / dx), periodic.
"""
import math

M_H = 1.6735575e-24   # g


def boost(t, a_b, k_b):
    return max(1.0, a_b * math.exp(k_b / t)) if a_b > 0 else 1.0


def emitting_time(age, lifetime, interval):
    a_p = age - interval
    if a_p >= lifetime:
        return 0.0
    if a_p < 0:
        return min(age, lifetime)
    return min(interval, lifetime - a_p)


def star_rate(star, interval, f_esc=1.0, a_b=0.0, k_b=0.0, t_universe=1.0):
    """Effective emission rate [photons/s] of one star (a mapping with mass, age, lifetime,
    photons_per_baryon) over the interval."""
    ndot = star["photons_per_baryon"] * star["mass"] / M_H / star["lifetime"]
    e = emitting_time(star["age"], star["lifetime"], interval)
    return e / interval * ndot * f_esc * boost(t_universe, a_b, k_b)


def star_cell(star, shape, dx):
    nz, ny, nx = shape
    i = math.floor(star["x"] / dx) % nx
    j = math.floor(star["y"] / dx) % ny
    k = math.floor(star["z"] / dx) % nz
    return i + nx * (j + ny * k)


def star_sources(stars, shape, dx, interval, **model):
    """(cells, rates) lists in star order; cell -1 and rate 0 for stars that are not active
    inside the interval (zero emitting time)."""
    cells, rates = [], []
    for s in stars:
        if emitting_time(s["age"], s["lifetime"], interval) > 0:
            cells.append(star_cell(s, shape, dx))
            rates.append(star_rate(s, interval, **model))
        else:
            cells.append(-1)
            rates.append(0.0)
    return cells, rates

"""Snapshot-sequence post-processing driver (section 2.3): for each interval between two
snapshots, the star list of the later snapshot becomes nearest-grid-point emission rates
(aton_star_sources: lifetime dilution, escape fraction, boost factor), which replace the
handle's sources (aton_add_sources), and the handle advances by the interval's steps. Every
computation runs in libaton.so; this module only orders the calls.
"""
import numpy as np

from . import aton as A


def run_snapshots(a, snapshots, shape, dx, dt, interval, f_esc=1.0, boost_a=0.0, boost_k=0.0,
                  t0=0.0, stats=False):
    """Post-process the intervals between consecutive snapshots on handle `a`.

    The interval is covered by K = round(interval / dt) steps; the rates are scaled by
    interval / (K dt) so the photons each interval emits are exactly the model's. The boost is
    evaluated at the interval's mid time t0 + (p + 1/2) interval. Returns one record per
    interval: the number of emitting stars and cells, the photons the model emits, and (with
    stats) the ionisation statistics after the interval.
    """
    K = max(1, int(round(interval / dt)))
    scale = interval / (K * dt)
    out = []
    for p in range(len(snapshots) - 1):
        t_mid = t0 + (p + 0.5) * interval
        cell, rate = A.star_sources(snapshots[p + 1], shape, dx, interval, f_esc, boost_a,
                                    boost_k, t_mid)
        on = cell >= 0
        a.add_sources(cell[on], rate[on] * scale, A.SRC_REPLACE)
        a.step(K)
        rec = dict(interval=p, steps=K, stars=int(on.sum()), cells=int(np.unique(cell[on]).size),
                   photons=float(rate[on].sum() * interval), cell=cell[on], rate=rate[on] * scale)
        if stats:
            rec["stats"] = a.ionisation_stats()
        out.append(rec)
    return out

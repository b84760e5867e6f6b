"""Whole-step pins of the oracle: photon conservation (emitted = stored + absorbed + escaped +
clipped), the ionised-atom count, and the Stromgren sphere of a point source in a uniform
medium, r(t) = r_S (1 - exp(-t/t_rec))^(1/3)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1004_2503_b300 import workloads as W

C = W.C_LIGHT


def _params(run, **kw):
    bc = O.BC_TRANSMISSIVE if run["bc"] == "transmissive" else O.BC_PERIODIC
    base = dict(c=run["c"], dx=run["dx"], dt=run["dt"], sigma_n=run["sigma_n"],
                sigma_e=run["sigma_e"], e_gamma_eV=run["e_gamma_eV"], bc=bc)
    base.update(kw)
    return O.params(**base)


def _closure(p, st0, st1, b):
    s0 = O.stored(p, st0["N"])
    s1 = O.stored(p, st1["N"])
    return (s0 + b["emitted"]) - (s1 + b["absorbed"] + b["escaped"] + b["clipped"])


def test_budget_identity_periodic_lognormal():
    st, idx, rate, run = W.workload_small()
    p = _params(run)
    out, b, s = O.run(p, st, 30, idx, rate)
    assert b["emitted"] > 0 and b["absorbed"] > 0
    assert abs(_closure(p, st, out, b)) <= 1e-12 * b["emitted"]
    assert b["escaped"] == 0.0 and s["error_cells"] == 0


def test_budget_identity_transmissive_with_escape():
    st, idx, rate, run = W.stromgren_box(n=16, L_kpc=1.0, nH=1e-5, x0=0.5)
    p = _params(run, fixed_T=0)
    out, b, s = O.run(p, st, 120, idx, rate)
    assert b["escaped"] > 0.01 * b["emitted"]
    assert abs(_closure(p, st, out, b)) <= 1e-12 * b["emitted"]


def test_32_cube_ionised_atoms_equal_absorbed_photons():
    """Uniform 32^3 box, one 5e48 /s source, T fixed at 1e4 K, no collisional ionisation,
    500 steps (t << t_rec): every absorbed photon ionised one atom, less a small number of
    recombinations."""
    st, idx, rate, run = W.workload_32()
    p = _params(run, fixed_T=1, coll_ion=0)
    out, b, s = O.run(p, st, 500, idx, rate, omp=True)
    V = run["dx"] ** 3
    ionised = float(np.sum(out["nH"] * (out["x"] - st["x"])) * V)
    assert b["absorbed"] > 0.5 * b["emitted"]
    rel = (b["absorbed"] - ionised) / b["absorbed"]
    assert 0.0 <= rel < 2e-3
    assert abs(_closure(p, st, out, b)) <= 1e-12 * b["emitted"]
    assert s["error_cells"] == 0


@pytest.mark.slow
def test_stromgren_sphere_radius_and_balance():
    """nH = 1 cm^-3, T = 1e4 K fixed, Ndot = 5e48 /s: r_S = (3 Ndot / (4 pi alpha_B nH^2))^(1/3)
    with the textbook alpha_B(1e4 K) = 2.59e-13. A reduced speed of light (c/100) keeps the
    run short; it changes neither r_S nor the approach r(t) once t >> r_S / c.

    Checks: the ionised-volume radius follows r_S (1 - e^{-t/t_rec})^{1/3} within one cell at
    t = 1, 2, 4 t_rec, and at late time the recombination volume sum(x^2) V balances the
    source, sum(x^2) V = 4/3 pi r_S^3, within 2 %."""
    n, T, Ndot = 1.0, 1e4, 5e48
    aB = 2.59e-13
    rS = (3 * Ndot / (4 * math.pi * aB * n * n)) ** (1 / 3)
    trec = 1.0 / (aB * n)
    ncell = 20
    dx = rS / 6.0
    c = C / 100.0
    st, idx, rate, run = W.stromgren_box(n=ncell, L_kpc=ncell * dx / W.KPC, nH=n, T0=T,
                                         x0=1.2e-3, rate=Ndot, c=c)
    p = _params(run, fixed_T=1, coll_ion=0)
    V = dx ** 3
    steps_per_trec = trec / run["dt"]
    budget, stats = None, None
    t_done = 0
    cur = st
    for k in (1, 2, 4, 7):
        nsteps = int(round(k * steps_per_trec)) - t_done
        cur, budget, stats = O.run(p, cur, nsteps, idx, rate, omp=True, budget=budget,
                                   stats=stats)
        t_done += nsteps
        t = t_done * run["dt"]
        if k <= 4:
            r_eff = (3 * np.sum(cur["x"] - st["x"]) * V / (4 * math.pi)) ** (1 / 3)
            r_th = rS * (1 - math.exp(-t / trec)) ** (1 / 3)
            assert abs(r_eff - r_th) < dx, (k, r_eff / dx, r_th / dx)
    vol = float(np.sum(cur["x"] ** 2) * V)
    assert vol == pytest.approx(4 * math.pi / 3 * rS ** 3, rel=0.02)
    assert budget["escaped"] < 1e-3 * budget["emitted"]

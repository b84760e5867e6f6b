"""The oracle's one-cell step (used to check sampled cells of grids too large for a whole-grid
oracle run) is the whole-grid step restricted to one cell: transport of the centre from its
3x3x3 neighbourhood with the intercell flux (Appendix Eq. A2 in 3-D, Eq. A5), the
realisability clamp, the cell's sources (section 2.3) and the operator Phi (Eq. A4).

Checked cell by cell against ``orc_step`` on a periodic lognormal box with sources and on a
transmissive Stromgren box (ghost = copy of the boundary cell), with both intercell fluxes.
The neighbourhoods are cut here with numpy (wrap or edge padding), independently of any
helper the GPU tests use.
"""
import numpy as np
import pytest

import oracle as O
from paper_1004_2503_b300 import workloads as W

FIELDS = ("N", "Fx", "Fy", "Fz")


def _params(run, **kw):
    bc = O.BC_TRANSMISSIVE if run["bc"] == "transmissive" else O.BC_PERIODIC
    base = dict(c=run["c"], dx=run["dx"], dt=run["dt"], sigma_n=run["sigma_n"],
                sigma_e=run["sigma_e"], e_gamma_eV=run["e_gamma_eV"], bc=bc)
    base.update(kw)
    return O.params(**base)


def _compare_every_cell(p, st, idx, rate, periodic):
    after, _, _ = O.run(p, st, 1, idx, rate)
    shape = st["N"].shape
    cell_rate = np.bincount(np.asarray(idx, np.int64), weights=np.asarray(rate, np.float64),
                            minlength=st["N"].size).reshape(shape)
    mode = "wrap" if periodic else "edge"
    pad = {q: np.pad(np.asarray(st[q], np.float64), 1, mode=mode) for q in FIELDS}
    worst = 0.0
    for k in range(shape[0]):
        for j in range(shape[1]):
            for i in range(shape[2]):
                nb = [pad[q][k:k + 3, j:j + 3, i:i + 3] for q in FIELDS]
                r = O.cell_step(p, *nb, st["x"][k, j, i], st["T"][k, j, i], st["nH"][k, j, i],
                                cell_rate[k, j, i])
                assert r["err"] == 0
                for q in ("N", "Fx", "Fy", "Fz", "x", "T"):
                    a, b = r[q], after[q][k, j, i]
                    d = abs(a - b) / max(abs(b), 1e-300) if b != 0 else abs(a)
                    worst = max(worst, d)
    return worst


def _evolved(st, idx, rate, p, nsteps):
    out, _, _ = O.run(p, st, nsteps, idx, rate)
    return out


@pytest.mark.parametrize("flux", [O.FLUX_GLF, O.FLUX_HLL])
def test_cell_step_equals_the_grid_step_on_a_periodic_box_with_sources(flux):
    st, idx, rate, run = W.workload_small(shape=(8, 10, 12), nsrc=5)
    assert len(set(np.asarray(idx).tolist())) == len(idx)   # one source per cell
    p = _params(run, flux=flux)
    st = _evolved(st, idx, rate, p, 6)    # a radiation field with flux in every direction
    assert np.count_nonzero(st["N"]) > 0.5 * st["N"].size
    assert _compare_every_cell(p, st, idx, rate, periodic=True) <= 1e-14


@pytest.mark.parametrize("flux", [O.FLUX_GLF, O.FLUX_HLL])
def test_cell_step_equals_the_grid_step_on_a_transmissive_box(flux):
    st, idx, rate, run = W.stromgren_box(n=9, L_kpc=1.0, nH=1e-4, x0=0.2)
    p = _params(run, flux=flux, fixed_T=0)
    st = _evolved(st, idx, rate, p, 12)   # the front has reached the faces
    edge = np.concatenate([st["N"][0].ravel(), st["N"][-1].ravel()])
    assert edge.max() > 0
    assert _compare_every_cell(p, st, idx, rate, periodic=False) <= 1e-14

"""Helpers shared by the GPU parity tests: run a workload through the C ABI and through the
oracle, and measure their differences with the accuracy gates used throughout:
  x: absolute difference <= 1e-3
  T: relative difference <= 1e-3
  N: relative difference <= 1e-3 on cells with N > 1e-6 max N
"""
import numpy as np

import oracle as O
from paper_1004_2503_b300 import aton as A

TOL_X = 1e-3
TOL_T = 1e-3
TOL_N = 1e-3
N_FLOOR = 1e-6


def oracle_params(run, **kw):
    bc = O.BC_TRANSMISSIVE if run["bc"] == "transmissive" else O.BC_PERIODIC
    base = dict(c=run["c"], dx=run["dx"], dt=run["dt"], sigma_n=run["sigma_n"],
                sigma_e=run["sigma_e"], e_gamma_eV=run["e_gamma_eV"], bc=bc)
    base.update(kw)
    return O.params(**base)


def run_oracle(state, idx, rate, run, nsteps, omp=True, **kw):
    p = oracle_params(run, **kw)
    out, b, s = O.run(p, state, nsteps, idx, rate, omp=omp)
    b = dict(b)
    b["stored0"] = O.stored(p, state["N"])
    b["stored"] = O.stored(p, out["N"])
    return out, b, s


def run_gpu(state, idx, rate, run, nsteps, mode=A.MODE_FUSED, graph_batch=100, tile=None,
            rows=None, **kw):
    a = A.from_workload(state, idx, rate, run, **kw)
    try:
        a.set_exec(mode, graph_batch)
        if tile is not None:
            a.set_tile(*tile)
        if rows is not None:
            a.set_tile_rows(rows)
        a.step(nsteps)
        rc = a.synchronize()
        f = a.get_fields()
        b = a.photon_budget()
        d = a.diag()
    finally:
        a.close()
    return f, b, d, rc


def errors(gpu, orc):
    """Per-field errors of the GPU state against the oracle state."""
    xg = gpu["x"].astype(np.float64)
    e = {}
    e["x_abs"] = float(np.abs(xg - orc["x"]).max())
    e["y_rel_ionised"] = float(np.max(np.abs(gpu["y"] - (1 - orc["x"])) /
                                      np.maximum(1 - orc["x"], 1e-6)))
    e["T_rel"] = float(np.max(np.abs(gpu["T"] - orc["T"]) / orc["T"]))
    No = orc["N"]
    mask = No > N_FLOOR * No.max() if No.max() > 0 else np.zeros_like(No, bool)
    e["N_rel"] = float(np.max(np.abs(gpu["N"][mask] - No[mask]) / No[mask])) if mask.any() else 0.0
    e["N_l1_rel"] = float(np.abs(gpu["N"] - No).sum() / max(np.abs(No).sum(), 1e-300))
    Fo = np.sqrt(orc["Fx"] ** 2 + orc["Fy"] ** 2 + orc["Fz"] ** 2)
    dF = np.sqrt((gpu["Fx"] - orc["Fx"]) ** 2 + (gpu["Fy"] - orc["Fy"]) ** 2 +
                 (gpu["Fz"] - orc["Fz"]) ** 2)
    c = 2.99792458e10
    e["F_rel_cN"] = float(np.max(dF[mask] / (c * No[mask]))) if mask.any() else 0.0
    return e


def assert_gates(e, tag=""):
    assert e["x_abs"] <= TOL_X, (tag, e)
    assert e["T_rel"] <= TOL_T, (tag, e)
    assert e["N_rel"] <= TOL_N, (tag, e)


def budget_closure(b):
    lhs = b["stored0"] + b["emitted"]
    rhs = b["stored"] + b["absorbed"] + b["escaped"] + b["clipped"]
    return (lhs - rhs) / max(b["emitted"], 1e-300)


def neighbourhood(fields, cell, shape, periodic):
    """3x3x3 ghost-filled neighbourhood of ``cell`` (periodic wrap or transmissive copy)."""
    nz, ny, nx = shape
    k, j, i = np.unravel_index(int(cell), shape)

    def m(v, n):
        if periodic:
            return v % n
        return min(max(v, 0), n - 1)
    ks = [m(k - 1, nz), k, m(k + 1, nz)]
    js = [m(j - 1, ny), j, m(j + 1, ny)]
    is_ = [m(i - 1, nx), i, m(i + 1, nx)]
    sl = np.ix_(ks, js, is_)
    return {q: np.asarray(fields[q][sl], np.float64) for q in ("N", "Fx", "Fy", "Fz")}, (k, j, i)

"""Parity at the full 512^3 workload in the launch configuration the benchmark times
(autotuned fused kernel, CUDA graphs), on sampled cells: the oracle takes one step of each
sampled cell from its 3x3x3 neighbourhood in the GPU's previous state. Plus the photon budget
identity, which holds at any size."""
import numpy as np
import pytest

import oracle as O
from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import workloads as W

from parity_helpers import neighbourhood, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w512():
    return W.workload_512()


def test_512_sampled_cells_match_the_oracle_step(w512):
    st, idx, rate, run = w512
    shape = st["N"].shape
    a = A.from_workload(st, idx, rate, run)
    a.autotune(1)
    a.set_exec(a.get_exec()["mode"], 100)
    a.step(20)                       # let fronts form around the sources
    prev = a.get_fields()
    a.step(1)
    assert a.synchronize() == 0
    cur = a.get_fields()
    b = a.photon_budget()
    a.close()
    clos = (b["stored0"] + b["emitted"] - b["stored"] - b["absorbed"] - b["escaped"] -
            b["clipped"]) / b["emitted"]
    assert abs(clos) <= 1e-6
    p = oracle_params(run)
    src = dict(zip(idx.tolist(), rate.tolist()))
    rng = np.random.default_rng(0)
    hot = np.argsort(prev["N"].ravel())[-64:]               # brightest cells (sources, fronts)
    sample = np.unique(np.concatenate([idx[:64], hot, rng.choice(prev["N"].size, 128, replace=False)]))
    worst = dict(x=0.0, T=0.0, N=0.0)
    for cell in sample:
        nb, (k, j, i) = neighbourhood(prev, cell, shape, periodic=True)
        r = O.cell_step(p, nb["N"], nb["Fx"], nb["Fy"], nb["Fz"], float(prev["x"][k, j, i]),
                        float(prev["T"][k, j, i]), float(st["nH"][k, j, i]), src.get(int(cell), 0.0))
        worst["x"] = max(worst["x"], abs(float(cur["x"][k, j, i]) - r["x"]))
        worst["T"] = max(worst["T"], abs(float(cur["T"][k, j, i]) - r["T"]) / r["T"])
        if r["N"] > 1e-6 * float(prev["N"].max()):
            worst["N"] = max(worst["N"], abs(float(cur["N"][k, j, i]) - r["N"]) / r["N"])
    print("512^3 sampled worst", worst, "cells", len(sample))
    assert worst["x"] <= 1e-3 and worst["T"] <= 1e-3 and worst["N"] <= 1e-3, worst


def test_1024_sampled_cells_match_the_oracle_step():
    """The 1024^3 workload (43 GB of float32 state on the device): one step of sampled cells
    against the oracle, after 10 steps in the benchmark's launch configuration."""
    st, idx, rate, run = W.workload_1024()
    shape = st["N"].shape
    a = A.from_workload(st, idx, rate, run)
    a.autotune(1)
    a.set_exec(a.get_exec()["mode"], 100)
    a.step(10)
    prev = a.get_fields()
    a.step(1)
    assert a.synchronize() == 0
    cur = a.get_fields()
    b = a.photon_budget()
    a.close()
    clos = (b["stored0"] + b["emitted"] - b["stored"] - b["absorbed"] - b["escaped"] -
            b["clipped"]) / b["emitted"]
    assert abs(clos) <= 1e-6
    p = oracle_params(run)
    src = dict(zip(idx.tolist(), rate.tolist()))
    rng = np.random.default_rng(1)
    hot = np.argpartition(prev["N"].ravel(), -64)[-64:]
    sample = np.unique(np.concatenate([idx[:64], hot, rng.choice(prev["N"].size, 128, replace=False)]))
    worst = dict(x=0.0, T=0.0, N=0.0)
    for cell in sample:
        nb, (k, j, i) = neighbourhood(prev, cell, shape, periodic=True)
        r = O.cell_step(p, nb["N"], nb["Fx"], nb["Fy"], nb["Fz"], float(prev["x"][k, j, i]),
                        float(prev["T"][k, j, i]), float(st["nH"][k, j, i]), src.get(int(cell), 0.0))
        worst["x"] = max(worst["x"], abs(float(cur["x"][k, j, i]) - r["x"]))
        worst["T"] = max(worst["T"], abs(float(cur["T"][k, j, i]) - r["T"]) / r["T"])
        if r["N"] > 1e-6 * float(prev["N"].max()):
            worst["N"] = max(worst["N"], abs(float(cur["N"][k, j, i]) - r["N"]) / r["N"])
    print("1024^3 sampled worst", worst, "cells", len(sample))
    assert worst["x"] <= 1e-3 and worst["T"] <= 1e-3 and worst["N"] <= 1e-3, worst
